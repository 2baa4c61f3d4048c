// The C ABI (include/mgc.h): argument checking, handle lifetime and dispatch
// to the kernels of the other translation units.
#include <atomic>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>

#include "mgc_host.h"

namespace mgc {

static thread_local std::string g_last_error;

int fail(int code, const std::string &msg)
{
    g_last_error = msg;
    return code;
}

int cuda_fail(cudaError_t e, const char *what, const char *file, int line)
{
    char buf[512];
    snprintf(buf, sizeof(buf), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file, line);
    g_last_error = buf;
    // clear the runtime's last-error state so that a later launch check does
    // not report this (non-sticky) error again
    (void)cudaGetLastError();
    return MGC_ERR_CUDA;
}

int ok() { return MGC_OK; }

int check_device_status(const mgc_clover_s *op, cudaStream_t s)
{
    int h = 0;
    MGC_CUDA(cudaMemcpyAsync(&h, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    if (h) {
        MGC_CUDA(cudaMemsetAsync(op->d_status, 0, sizeof(int), s));
        return fail(MGC_ERR_TIMEOUT, "a bounded device wait in the smoother ran out");
    }
    return MGC_OK;
}

static std::atomic<long long> g_launches{0};
static std::atomic<long long> g_bytes{0};

void count(long long launches, double bytes)
{
    g_launches += launches;
    g_bytes += (long long)bytes;
}

double spinor_site_bytes(int prec) { return prec == 64 ? 192.0 : (prec == 32 ? 96.0 : 52.0); }

double links_site_bytes(int prec, int compress)
{
    const double reals = (prec == 64 || compress == 18) ? 18.0 : 12.0;
    return 4.0 * reals * (prec == 64 ? 8.0 : (prec == 32 ? 4.0 : 2.0));
}

double clover_site_bytes(int prec) { return prec == 64 ? 576.0 : (prec == 32 ? 288.0 : 148.0); }

static int ilog2(int v)
{
    int l = 0;
    while ((1 << l) < v) ++l;
    return ((1 << l) == v) ? l : -1;
}

}  // namespace mgc

using namespace mgc;

extern "C" {

int mgc_version(void) { return 10000; }

const char *mgc_status_string(int status)
{
    switch (status) {
    case MGC_OK: return "MGC_OK";
    case MGC_ERR_INVALID_ARG: return "MGC_ERR_INVALID_ARG";
    case MGC_ERR_UNSUPPORTED_SHAPE: return "MGC_ERR_UNSUPPORTED_SHAPE";
    case MGC_ERR_NOT_UNITARY: return "MGC_ERR_NOT_UNITARY";
    case MGC_ERR_CUDA: return "MGC_ERR_CUDA";
    case MGC_NOT_CONVERGED: return "MGC_NOT_CONVERGED";
    case MGC_ERR_BREAKDOWN: return "MGC_ERR_BREAKDOWN";
    case MGC_ERR_TIMEOUT: return "MGC_ERR_TIMEOUT";
    case MGC_ERR_NO_DEVICE: return "MGC_ERR_NO_DEVICE";
    default: return "MGC_UNKNOWN_STATUS";
    }
}

const char *mgc_last_error(void) { return g_last_error.c_str(); }

int mgc_counters(long long *launches, double *algorithmic_bytes, int reset)
{
    if (launches) *launches = g_launches.load();
    if (algorithmic_bytes) *algorithmic_bytes = (double)g_bytes.load();
    if (reset) {
        g_launches = 0;
        g_bytes = 0;
    }
    return MGC_OK;
}

int mgc_lattice_create(const int dims[4], const int block[4], int t_bc, mgc_lattice_t *out)
{
    if (!dims || !block || !out) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    if (t_bc != 1 && t_bc != -1) return fail(MGC_ERR_INVALID_ARG, "t_bc must be +1 or -1");
    Geom g{};
    long long V = 1;
    int lvb = 0;
    for (int mu = 0; mu < 4; ++mu) {
        const int lb = ilog2(block[mu]);
        if (dims[mu] < 1 || lb < 1) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "block extents must be powers of two >= 2");
        if (dims[mu] % block[mu] != 0) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "lattice extent not divisible by block");
        const int nb = dims[mu] / block[mu];
        if (nb % 2 != 0) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "blocks per direction must be even");
        g.L[mu] = dims[mu];
        g.NB[mu] = nb;
        g.lb[mu] = lb;
        lvb += lb;
        V *= dims[mu];
    }
    if (lvb > 10) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "at most 1024 sites per block");
    if (V > (1LL << 30)) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "lattice too large (> 2^30 sites)");
    g.lvb = lvb;
    g.V = (int)V;
    g.nblocks = g.NB[0] * g.NB[1] * g.NB[2] * g.NB[3];
    g.tbc = t_bc;
    mgc_lattice_s *L = new mgc_lattice_s();
    L->g = g;
    for (int mu = 0; mu < 4; ++mu) {
        L->dims[mu] = dims[mu];
        L->block[mu] = block[mu];
    }
    *out = L;
    return MGC_OK;
}

int mgc_lattice_destroy(mgc_lattice_t lat)
{
    delete lat;
    return MGC_OK;
}

long long mgc_lattice_volume(mgc_lattice_t lat) { return lat ? (long long)lat->g.V : -1; }

size_t mgc_spinor_bytes(mgc_lattice_t lat, int prec, int nrhs)
{
    if (!lat || (prec != 64 && prec != 32 && prec != 16) || nrhs < 1) return 0;
    return spinor_bytes(lat->g, prec, nrhs);
}

static bool valid_prec(int p) { return p == 64 || p == 32 || p == 16; }

int mgc_spinor_pack(mgc_lattice_t lat, int prec, int nrhs, const double *canonical, void *packed, void *stream)
{
    if (!lat || !canonical || !packed || !valid_prec(prec) || nrhs < 1) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return launch_pack(lat->g, prec, nrhs, canonical, packed, (cudaStream_t)stream);
}

int mgc_spinor_unpack(mgc_lattice_t lat, int prec, int nrhs, const void *packed, double *canonical, void *stream)
{
    if (!lat || !canonical || !packed || !valid_prec(prec) || nrhs < 1) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return launch_unpack(lat->g, prec, nrhs, packed, canonical, (cudaStream_t)stream);
}

int mgc_spinor_convert(mgc_lattice_t lat, int nrhs, int prec_in, const void *in, int prec_out, void *out, void *stream)
{
    if (!lat || !in || !out || !valid_prec(prec_in) || !valid_prec(prec_out) || nrhs < 1 || in == out)
        return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return launch_convert(lat->g, nrhs, prec_in, in, prec_out, out, (cudaStream_t)stream);
}

int mgc_gauge_create(mgc_lattice_t lat, const double *U, int on_device, int storage_prec, int compress, void *stream,
                     mgc_gauge_t *out)
{
    if (!lat || !U || !out || !valid_prec(storage_prec) || (compress != 18 && compress != 12))
        return fail(MGC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Geom &g = lat->g;
    const size_t cb = (size_t)g.V * 4 * 9 * 16;
    double *canon = nullptr;
    mgc_gauge_s *G = new mgc_gauge_s();
    G->lat = lat;
    G->prec = storage_prec;
    G->compress = (storage_prec == 64) ? 18 : compress;
    int st = MGC_OK;
    double *d_err = nullptr;
    auto bail = [&](int code) {
        cudaFree(canon);
        cudaFree(d_err);
        if (code != MGC_OK) {
            cudaFree(G->U64);
            cudaFree(G->U32);
            cudaFree(G->U16);
            delete G;
        }
        return code;
    };
#define GCUDA(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call, __FILE__, __LINE__)); \
    } while (0)
    const double *src = U;
    if (!on_device) {
        GCUDA(cudaMalloc(&canon, cb));
        GCUDA(cudaMemcpyAsync(canon, U, cb, cudaMemcpyHostToDevice, s));
        src = canon;
    }
    if (G->compress == 12) {
        GCUDA(cudaMalloc(&d_err, sizeof(double)));
        GCUDA(cudaMemsetAsync(d_err, 0, sizeof(double), s));
        st = launch_unitarity(g, src, d_err, s);
        if (st) return bail(st);
        double h = 0;
        GCUDA(cudaMemcpyAsync(&h, d_err, sizeof(double), cudaMemcpyDeviceToHost, s));
        GCUDA(cudaStreamSynchronize(s));
        if (!(h <= 1e-10)) return bail(fail(MGC_ERR_NOT_UNITARY, "12-real compression needs SU(3) links"));
    }
    GCUDA(cudaMalloc(&G->U64, gauge_bytes(g, 64, 18)));
    st = launch_gauge_pack(g, src, 64, 18, G->U64, s);
    if (st) return bail(st);
    if (storage_prec <= 32) {
        GCUDA(cudaMalloc(&G->U32, gauge_bytes(g, 32, G->compress)));
        st = launch_gauge_pack(g, src, 32, G->compress, G->U32, s);
        if (st) return bail(st);
    }
    if (storage_prec == 16) {
        GCUDA(cudaMalloc(&G->U16, gauge_bytes(g, 16, G->compress)));
        st = launch_gauge_pack(g, src, 16, G->compress, G->U16, s);
        if (st) return bail(st);
    }
    GCUDA(cudaStreamSynchronize(s));
#undef GCUDA
    *out = G;
    return bail(MGC_OK);
}

int mgc_gauge_destroy(mgc_gauge_t g)
{
    if (!g) return MGC_OK;
    cudaFree(g->U64);
    cudaFree(g->U32);
    cudaFree(g->U16);
    delete g;
    return MGC_OK;
}

int mgc_clover_create(mgc_gauge_t g, double kappa, double csw, void *stream, mgc_clover_t *out)
{
    if (!g || !out) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const Geom &geo = g->lat->g;
    mgc_clover_s *op = new mgc_clover_s();
    op->gauge = g;
    op->kappa = kappa;
    op->csw = csw;
    int *d_bad = nullptr;
    auto bail = [&](int code) {
        cudaFree(d_bad);
        if (code != MGC_OK) {
            cudaFree(op->C64);
            cudaFree(op->Ci64);
            cudaFree(op->C32);
            cudaFree(op->C16);
            cudaFree(op->Ci32);
            cudaFree(op->Ci16);
            cudaFree(op->d_status);
            delete op;
        }
        return code;
    };
#define CCUDA(call)                                                                   \
    do {                                                                              \
        cudaError_t e_ = (call);                                                      \
        if (e_ != cudaSuccess) return bail(cuda_fail(e_, #call, __FILE__, __LINE__)); \
    } while (0)
    CCUDA(cudaMalloc(&op->d_status, sizeof(int)));
    CCUDA(cudaMemsetAsync(op->d_status, 0, sizeof(int), s));
    CCUDA(cudaMalloc(&op->C64, clover_bytes(geo, 64)));
    CCUDA(cudaMalloc(&op->Ci64, clover_bytes(geo, 64)));
    CCUDA(cudaMalloc(&d_bad, sizeof(int)));
    CCUDA(cudaMemsetAsync(d_bad, 0, sizeof(int), s));
    int st = launch_clover_build(geo, g->U64, kappa, csw, op->C64, op->Ci64, d_bad, s);
    if (st) return bail(st);
    // C and C^-1 (the latter for the clover-preconditioned operator A = C^-1 D)
    // at every precision the gauge field keeps
    if (g->prec <= 32) {
        CCUDA(cudaMalloc(&op->C32, clover_bytes(geo, 32)));
        st = launch_clover_lowprec(geo, op->C64, 32, op->C32, s);
        if (st) return bail(st);
        CCUDA(cudaMalloc(&op->Ci32, clover_bytes(geo, 32)));
        st = launch_clover_lowprec(geo, op->Ci64, 32, op->Ci32, s);
        if (st) return bail(st);
    }
    if (g->prec == 16) {
        CCUDA(cudaMalloc(&op->C16, clover_bytes(geo, 16)));
        op->C16_sc = (float *)((uint4 *)op->C16 + (size_t)geo.V * 9);
        st = launch_clover_lowprec(geo, op->C64, 16, op->C16, s);
        if (st) return bail(st);
        CCUDA(cudaMalloc(&op->Ci16, clover_bytes(geo, 16)));
        op->Ci16_sc = (float *)((uint4 *)op->Ci16 + (size_t)geo.V * 9);
        st = launch_clover_lowprec(geo, op->Ci64, 16, op->Ci16, s);
        if (st) return bail(st);
    }
    int bad = 0;
    CCUDA(cudaMemcpyAsync(&bad, d_bad, sizeof(int), cudaMemcpyDeviceToHost, s));
    CCUDA(cudaStreamSynchronize(s));
#undef CCUDA
    if (bad) return bail(fail(MGC_ERR_BREAKDOWN, "singular clover block"));
    *out = op;
    return bail(MGC_OK);
}

int mgc_clover_destroy(mgc_clover_t op)
{
    if (!op) return MGC_OK;
    free_work(op);
    cudaFree(op->C64);
    cudaFree(op->Ci64);
    cudaFree(op->C32);
    cudaFree(op->C16);
    cudaFree(op->Ci32);
    cudaFree(op->Ci16);
    cudaFree(op->d_status);
    delete op;
    return MGC_OK;
}

int mgc_selftest_bounded_wait(long long limit_ns, int arrive, int *flag_out, void *stream)
{
    if (!flag_out || limit_ns <= 0 || limit_ns > 2000000000LL) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return selftest_bounded_wait(limit_ns, arrive, flag_out, (cudaStream_t)stream);
}

int mgc_fma_peak(int prec, double *flops_per_s, void *stream)
{
    if (!flops_per_s) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    return fma_peak(prec, flops_per_s, (cudaStream_t)stream);
}

int mgc_device_status(mgc_clover_t op, int *flags, int clear, void *stream)
{
    if (!op || !flags) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    MGC_CUDA(cudaMemcpyAsync(flags, op->d_status, sizeof(int), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    if (clear) MGC_CUDA(cudaMemsetAsync(op->d_status, 0, sizeof(int), s));
    return *flags ? fail(MGC_ERR_TIMEOUT, "a bounded device wait ran out") : MGC_OK;
}

int mgc_clover_export(mgc_clover_t op, int inverse, double *out, void *stream)
{
    if (!op || !out) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    return launch_clover_export(op->gauge->lat->g, inverse ? op->Ci64 : op->C64, out, (cudaStream_t)stream);
}

static int check_apply(mgc_clover_t op, const void *in, void *out, int nrhs, int prec)
{
    if (!op || !in || !out || nrhs < 1 || !valid_prec(prec)) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    if (in == out) return fail(MGC_ERR_INVALID_ARG, "in and out must not overlap");
    return MGC_OK;
}

int mgc_apply_D(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, void *stream)
{
    MGC_TRY(check_apply(op, in, out, nrhs, prec));
    return launch_dirac(op, prec, false, in, out, nrhs, (cudaStream_t)stream);
}

int mgc_apply_Ddag(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, void *stream)
{
    MGC_TRY(check_apply(op, in, out, nrhs, prec));
    return launch_dirac(op, prec, true, in, out, nrhs, (cudaStream_t)stream);
}

int mgc_apply_clover(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, int inverse, void *stream)
{
    MGC_TRY(check_apply(op, in, out, nrhs, prec));
    return launch_clover_apply(op, prec, inverse != 0, in, out, nrhs, (cudaStream_t)stream);
}

int mgc_sap_smooth(mgc_clover_t op, const void *b, void *x, int nrhs, int n_cy, int n_mr, int prec, int x_is_zero,
                   void *stream)
{
    MGC_TRY(check_apply(op, b, x, nrhs, prec));
    if (n_cy < 0 || n_mr < 0) return fail(MGC_ERR_INVALID_ARG, "n_cy and n_mr must be >= 0");
    return launch_sap(op, prec, b, x, nrhs, n_cy, n_mr, x_is_zero, (cudaStream_t)stream);
}

int mgc_sap_smooth_eo(mgc_clover_t op, const void *b, void *x, int nrhs, int n_cy, int n_mr, int prec,
                      int x_is_zero, void *stream)
{
    MGC_TRY(check_apply(op, b, x, nrhs, prec));
    if (n_cy < 0 || n_mr < 0) return fail(MGC_ERR_INVALID_ARG, "n_cy and n_mr must be >= 0");
    return launch_sap_eo(op, prec, b, x, nrhs, n_cy, n_mr, x_is_zero, (cudaStream_t)stream);
}

int mgc_apply_A(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, void *stream)
{
    MGC_TRY(check_apply(op, in, out, nrhs, prec));
    return launch_apply_A(op, prec, in, out, nrhs, (cudaStream_t)stream);
}

int mgc_sap_smooth_A(mgc_clover_t op, const void *b, void *x, int nrhs, int n_cy, int n_jacobi, int prec,
                     int x_is_zero, void *stream)
{
    MGC_TRY(check_apply(op, b, x, nrhs, prec));
    if (n_cy < 0 || n_jacobi < 0) return fail(MGC_ERR_INVALID_ARG, "n_cy and n_jacobi must be >= 0");
    return launch_sap_A(op, prec, b, x, nrhs, n_cy, n_jacobi, x_is_zero, (cudaStream_t)stream);
}

void mgc_solve_params_default(mgc_solve_params *p)
{
    if (!p) return;
    p->method = 2;
    p->precond = 1;
    p->smoother_prec = 32;
    p->n_cy = 4;
    p->n_mr = 4;
    p->restart = 16;
    p->tol = 1e-10;
    p->max_iter = 500;
    p->on_device = 1;
    p->x_is_guess = 0;
    p->inner_tol = 2e-6;
    p->sap_solver = 0;
}

int mgc_solve(mgc_clover_t op, const double *b, double *x, int nrhs, const mgc_solve_params *p, mgc_solve_info *info,
              void *stream)
{
    if (!op || !b || !x || !p || !info || nrhs < 1) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return mgc::solve(op, b, x, nrhs, p, info, (cudaStream_t)stream);
}

int mgc_solve_noalloc(mgc_clover_t op, const double *b, double *x, const mgc_solve_params *p, mgc_solve_info *info,
                      void *stream)
{
    if (!op || !b || !x || !p || !info) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return mgc::solve_noalloc(op, b, x, p, info, (cudaStream_t)stream);
}

int mgc_force(mgc_clover_t op, const double *phi, double *dSdU, const mgc_solve_params *p, mgc_solve_info *info,
              double *action, void *stream)
{
    if (!op || !phi || !dSdU || !p || !info) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    return mgc::force(op, phi, dSdU, p, info, action, (cudaStream_t)stream);
}

}  // extern "C"
