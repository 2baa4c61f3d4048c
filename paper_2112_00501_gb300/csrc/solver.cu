// FP64 flexible outer solvers around the SAP preconditioner (Sec. 3: the
// outer solver is flexible BiCGStab, the smoother is M_SAP), with every inner
// product, orthogonalisation and residual update in FP64 on the GPU.
//
//   FGCR(m): z_j = M r, w_j = D z_j, classical Gram-Schmidt of w_j against the
//   normalised w_0..w_{j-1} (the same combination applied to z_j), then
//   alpha = <w_j, r>, x += alpha z_j, r -= alpha w_j.  The residual is
//   recomputed as b - D x at the end of each cycle and when the recursive
//   residual meets the tolerance.
//   Flexible BiCGStab: the textbook recurrences with M applied to p and s.
//
// Reductions are deterministic: a fixed grid for a given vector length, a
// fixed per-thread element order, and a last-block pass that sums the block
// partials in a fixed order.  Scalars stay on the device; the host reads one
// residual norm per iteration.
#include <atomic>
#include <cmath>
#include <complex>
#include <cstdio>
#include <cstdlib>
#include <vector>

#include "mgc_host.h"

namespace mgc {

constexpr int RT = 256;        // reduction threads per block
constexpr int RGRID_MAX = 1024;
// accumulators one reduction block may deposit: the partial-sum area holds
// RGRID_MAX * PART_NV doubles, and every reduction template checks its width
constexpr int PART_NV = 32;
constexpr int MAXM = 32;

struct SolverWork {
    int m = 0;
    int lowprec = 0;
    double2 *x = nullptr, *r = nullptr, *b = nullptr, *t = nullptr;
    double2 *w[MAXM] = {}, *z[MAXM] = {};  // FGCR directions (BiCGStab reuses four of each)
    void *rl = nullptr, *zl = nullptr;
    float2 *r32 = nullptr;                  // two-level solve: FP32 inner vectors
    float2 *w32[MAXM] = {}, *z32[MAXM] = {};
    void *z16[MAXM] = {};                   // FP16 smoother outputs (FP16 smoother)
    int m32 = 0;
    double *scal = nullptr;     // device scalars
    double *partial = nullptr;  // reduction partials
    unsigned *counter = nullptr;
    double2 *stage = nullptr;   // canonical staging for host pointers
    double *hscal = nullptr;    // pinned host copy of a few scalars
    // host-pointer solves into page-locked x: the canonical x can go to the
    // host on copy_stream while the FP64 residual that confirms it is computed
    cudaStream_t copy_stream = nullptr;
    cudaEvent_t ev_x = nullptr, ev_copy = nullptr;
    double *host_x = nullptr;   // the caller's x of the current solve, else null
    bool copy_live = false;     // a copy of the current x to host_x is in flight
    // several host right-hand sides in page-locked memory: the next b crosses
    // the host link into stage2 (copy stream, ev_b) during the current solve
    double2 *stage2 = nullptr;
    cudaEvent_t ev_b = nullptr;
};

// device scalar slots
enum {
    S_BB = 0,      // ||b||^2
    S_RR = 1,      // ||r||^2
    S_NW = 2,      // ||w_j||^2 after orthogonalisation
    S_WR = 3,      // <w_j, r> (2 slots)
    S_RHO = 5,     // BiCGStab rho (2)
    S_R0V = 7,     // <r0, v> (2)
    S_TS = 9,      // <t, s> (2)
    S_TT = 11,     // <t, t>
    S_ALPHA = 14,  // BiCGStab alpha, omega, beta, formed once per iteration (2 slots each)
    S_OMEGA = 16,
    S_BETAB = 18,
    S_BETA = 32,   // CGS coefficients, 2 * MAXM slots
    S_TOTAL = 32 + 2 * MAXM,
};

__device__ __forceinline__ double2 cadd(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 csub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 cmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ double2 cdiv(double2 a, double2 b)
{
    const double n = b.x * b.x + b.y * b.y;
    return make_double2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n);
}
// conj(a) b accumulated into acc[0..1]
__device__ __forceinline__ void acc_dot(double *acc, double2 a, double2 b)
{
    acc[0] = fma(a.x, b.x, fma(a.y, b.y, acc[0]));
    acc[1] = fma(a.x, b.y, fma(-a.y, b.x, acc[1]));
}
__device__ __forceinline__ void acc_n2(double *acc, double2 a) { acc[0] = fma(a.x, a.x, fma(a.y, a.y, acc[0])); }
__device__ __forceinline__ double2 ld2(const double *p) { return make_double2(p[0], p[1]); }

template <int NV>
__device__ __forceinline__ void warp_reduce(double *v)
{
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
}

// sum NV values over the block; result valid on thread 0
template <int NV>
__device__ __forceinline__ void block_reduce(double *v, double (*sh)[RT / 32])
{
    warp_reduce<NV>(v);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0;
            for (int w = 0; w < RT / 32; ++w) s += sh[k][w];
            v[k] = s;
        }
    __syncthreads();
}

// out[k] = sum over elements e < n of the values f(e, acc) accumulates
template <int NV, class F>
__global__ void __launch_bounds__(RT) k_reduce(long long n, F f, double *partial, unsigned *counter, double *out)
{
    static_assert(NV <= PART_NV, "more accumulators than the partial-sum area holds");
    __shared__ double sh[NV][RT / 32];
    __shared__ bool last;
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0;
    for (long long e = (long long)blockIdx.x * RT + threadIdx.x; e < n; e += (long long)gridDim.x * RT) f(e, acc);
    block_reduce<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[blockIdx.x * NV + k] = acc[k];
        __threadfence();
        last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0;
    for (int bi = threadIdx.x; bi < (int)gridDim.x; bi += RT)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partial + bi * NV + k);
    block_reduce<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = acc[k];
        *counter = 0;
    }
}

// one thread forming scalars from scalars (no per-element FP64 divisions)
template <class F>
__global__ void k_scalar(F f)
{
    f();
}

template <class F>
static void scalar_step(F f, cudaStream_t s)
{
    k_scalar<<<1, 1, 0, s>>>(f);
    count(1, 0);
}

// a plain elementwise map
template <class F>
__global__ void __launch_bounds__(RT) k_map(long long n, F f)
{
    for (long long e = (long long)blockIdx.x * RT + threadIdx.x; e < n; e += (long long)gridDim.x * RT) f(e);
}

static int red_grid(long long n)
{
    long long g = (n + RT * 4 - 1) / (RT * 4);
    if (g > RGRID_MAX) g = RGRID_MAX;
    if (g < 1) g = 1;
    return (int)g;
}

// nvec: FP64 vectors of n complex entries the launch reads or writes
template <int NV, class F>
static int reduce(long long n, F f, SolverWork *W, double *out, cudaStream_t s, int nvec)
{
    k_reduce<NV><<<red_grid(n), RT, 0, s>>>(n, f, W->partial, W->counter, out);
    MGC_CUDA(cudaGetLastError());
    count(1, 16.0 * n * nvec);
    return MGC_OK;
}

template <class F>
static int map(long long n, F f, cudaStream_t s, int nvec)
{
    k_map<<<red_grid(n), RT, 0, s>>>(n, f);
    MGC_CUDA(cudaGetLastError());
    count(1, 16.0 * n * nvec);
    return MGC_OK;
}

struct PtrList {
    const double2 *p[MAXM];
};
struct MutPtrList {
    double2 *p[MAXM];
};

// ------------------------------------------------------------------ workspace
void free_work(mgc_clover_s *op)
{
    SolverWork *W = op->work;
    if (!W) return;
    cudaFree(W->x);
    cudaFree(W->r);
    cudaFree(W->b);
    cudaFree(W->t);
    for (auto p : W->w) cudaFree(p);
    for (auto p : W->z) cudaFree(p);
    cudaFree(W->rl);
    cudaFree(W->zl);
    cudaFree(W->r32);
    for (auto p : W->w32) cudaFree(p);
    for (auto p : W->z32) cudaFree(p);
    for (auto p : W->z16) cudaFree(p);
    cudaFree(W->scal);
    cudaFree(W->partial);
    cudaFree(W->counter);
    if (W->copy_stream) cudaStreamSynchronize(W->copy_stream);
    cudaFree(W->stage);
    cudaFree(W->stage2);
    cudaFreeHost(W->hscal);
    if (W->ev_x) cudaEventDestroy(W->ev_x);
    if (W->ev_copy) cudaEventDestroy(W->ev_copy);
    if (W->ev_b) cudaEventDestroy(W->ev_b);
    if (W->copy_stream) cudaStreamDestroy(W->copy_stream);
    delete W;
    op->work = nullptr;
}

// workspace for a method: FP64 Krylov vectors (methods 0, 1; BiCGStab needs
// four w and four z), FP32 Krylov vectors (method 2), smoother buffers at
// lowprec (16-bit smoother of the FP64 Krylov methods, or the FP16 smoother of
// the two-level solve)
static int ensure_work(mgc_clover_s *op, int method, int m, int lowprec)
{
    const Geom &g = op->gauge->lat->g;
    const int m64 = (method >= 2) ? 0 : (m < 4 ? 4 : m);
    const int m32 = (method == 2) ? m : (method == 3 ? 4 : 0);
    SolverWork *W = op->work;
    if (W && W->m >= m64 && W->m32 >= m32 && (lowprec == 64 || lowprec == 32 || W->lowprec == lowprec)) return MGC_OK;
    const int keep64 = W ? W->m : 0, keep32 = W ? W->m32 : 0, keeplow = W ? W->lowprec : 0;
    free_work(op);
    W = new SolverWork();
    op->work = W;
    const size_t vb = spinor_bytes(g, 64, 1);
    W->m = m64 > keep64 ? m64 : keep64;
    W->m32 = m32 > keep32 ? m32 : keep32;
    MGC_CUDA(cudaMalloc(&W->x, vb));
    MGC_CUDA(cudaMalloc(&W->r, vb));
    MGC_CUDA(cudaMalloc(&W->b, vb));
    MGC_CUDA(cudaMalloc(&W->t, vb));
    for (int j = 0; j < W->m; ++j) {
        MGC_CUDA(cudaMalloc(&W->w[j], vb));
        MGC_CUDA(cudaMalloc(&W->z[j], vb));
    }
    if (W->m32) {
        const size_t v32 = spinor_bytes(g, 32, 1);
        MGC_CUDA(cudaMalloc(&W->r32, v32));
        for (int j = 0; j < W->m32; ++j) {
            MGC_CUDA(cudaMalloc(&W->w32[j], v32));
            MGC_CUDA(cudaMalloc(&W->z32[j], v32));
        }
    }
    if (lowprec == 16 || keeplow == 16) {
        W->lowprec = 16;
        MGC_CUDA(cudaMalloc(&W->rl, spinor_bytes(g, 16, 1)));
        MGC_CUDA(cudaMalloc(&W->zl, spinor_bytes(g, 16, 1)));
        for (int j = 0; j < W->m32; ++j) MGC_CUDA(cudaMalloc(&W->z16[j], spinor_bytes(g, 16, 1)));
    } else if (lowprec == 32 || keeplow == 32) {
        W->lowprec = 32;
        MGC_CUDA(cudaMalloc(&W->rl, spinor_bytes(g, 32, 1)));
        MGC_CUDA(cudaMalloc(&W->zl, spinor_bytes(g, 32, 1)));
    }
    MGC_CUDA(cudaMalloc(&W->scal, S_TOTAL * sizeof(double)));
    MGC_CUDA(cudaMemset(W->scal, 0, S_TOTAL * sizeof(double)));
    MGC_CUDA(cudaMalloc(&W->partial, (size_t)RGRID_MAX * PART_NV * sizeof(double)));
    MGC_CUDA(cudaMalloc(&W->counter, sizeof(unsigned)));
    MGC_CUDA(cudaMemset(W->counter, 0, sizeof(unsigned)));
    MGC_CUDA(cudaMalloc(&W->stage, vb));
    MGC_CUDA(cudaMallocHost(&W->hscal, 2 * MAXM * sizeof(double)));
    MGC_CUDA(cudaStreamCreateWithFlags(&W->copy_stream, cudaStreamNonBlocking));
    MGC_CUDA(cudaEventCreateWithFlags(&W->ev_x, cudaEventDisableTiming));
    MGC_CUDA(cudaEventCreateWithFlags(&W->ev_copy, cudaEventDisableTiming));
    MGC_CUDA(cudaEventCreateWithFlags(&W->ev_b, cudaEventDisableTiming));
    return MGC_OK;
}

// x (canonical, through the staging buffer) to the caller's page-locked host
// x: the unpack on s, the copy on the copy stream, where it overlaps whatever
// s runs next
static int copy_x_early(mgc_clover_s *op, cudaStream_t s)
{
    SolverWork *W = op->work;
    const Geom &g = op->gauge->lat->g;
    MGC_TRY(launch_unpack(g, 64, 1, W->x, (double *)W->stage, s));
    MGC_CUDA(cudaEventRecord(W->ev_x, s));
    MGC_CUDA(cudaStreamWaitEvent(W->copy_stream, W->ev_x, 0));
    MGC_CUDA(cudaMemcpyAsync(W->host_x, W->stage, spinor_bytes(g, 64, 1), cudaMemcpyDeviceToHost, W->copy_stream));
    MGC_CUDA(cudaEventRecord(W->ev_copy, W->copy_stream));
    W->copy_live = true;
    return MGC_OK;
}

// s waits for an early copy of x: the staging buffer is free again and the
// host x complete once s reaches this point
static int join_copy(SolverWork *W, cudaStream_t s)
{
    if (!W->copy_live) return MGC_OK;
    W->copy_live = false;
    MGC_CUDA(cudaStreamWaitEvent(s, W->ev_copy, 0));
    return MGC_OK;
}

// page-locked host memory (a copy to pageable memory would not overlap)
static bool page_locked(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return false;
    }
    return a.type == cudaMemoryTypeHost;
}

// the smoother as preconditioner (x = 0 on entry), with the domain solver p->sap_solver
static int run_sap(mgc_clover_s *op, const mgc_solve_params *p, int prec, const void *v, void *z, cudaStream_t s)
{
    if (p->sap_solver == 2) return launch_sap_eo(op, prec, v, z, 1, p->n_cy, p->n_mr, 1, s);
    return launch_sap(op, prec, v, z, 1, p->n_cy, p->n_mr, 1, s);
}

// read one device scalar (synchronises the stream)
static int read_scalar(SolverWork *W, int slot, double *out, cudaStream_t s)
{
    MGC_CUDA(cudaMemcpyAsync(W->hscal, W->scal + slot, sizeof(double), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    *out = W->hscal[0];
    return MGC_OK;
}

// ------------------------------------------------------------------ building blocks
// z = M v (M = SAP in prec, or the identity)
static int precondition(mgc_clover_s *op, const mgc_solve_params *p, const double2 *v, double2 *z, cudaStream_t s)
{
    const Geom &g = op->gauge->lat->g;
    SolverWork *W = op->work;
    if (p->precond == 0) {
        MGC_CUDA(cudaMemcpyAsync(z, v, spinor_bytes(g, 64, 1), cudaMemcpyDeviceToDevice, s));
        return MGC_OK;
    }
    if (p->smoother_prec == 64) {
        MGC_CUDA(cudaMemsetAsync(z, 0, spinor_bytes(g, 64, 1), s));
        return run_sap(op, p, 64, v, z, s);
    }
    MGC_TRY(launch_convert(g, 1, 64, v, p->smoother_prec, W->rl, s));
    MGC_CUDA(cudaMemsetAsync(W->zl, 0, spinor_bytes(g, p->smoother_prec, 1), s));
    MGC_TRY(run_sap(op, p, p->smoother_prec, W->rl, W->zl, s));
    return launch_convert(g, 1, p->smoother_prec, W->zl, 64, z, s);
}

static int apply_D64(mgc_clover_s *op, const double2 *in, double2 *out, cudaStream_t s)
{
    return launch_dirac(op, 64, false, in, out, 1, s);
}

// r = b - t, and ||r||^2 into slot
static int residual(mgc_clover_s *op, double2 *r, const double2 *b, const double2 *t, int slot, cudaStream_t s)
{
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    return reduce<1>(
        n,
        [=] __device__(long long e, double *acc) {
            const double2 v = csub(b[e], t[e]);
            r[e] = v;
            acc_n2(acc, v);
        },
        W, W->scal + slot, s, 3);
}

static bool bad(double v) { return !std::isfinite(v); }

// ------------------------------------------------------------------ FGCR
static int fgcr(mgc_clover_s *op, const mgc_solve_params *p, mgc_solve_info *info, cudaStream_t s)
{
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    double2 *x = W->x, *r = W->r, *b = W->b, *t = W->t;
    double *sc = W->scal;
    const int m = p->restart;
    double bb, rr;

    MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, b[e]); }, W, sc + S_BB, s, 1));
    MGC_TRY(read_scalar(W, S_BB, &bb, s));
    info->iters = 0;
    info->restarts = 0;
    if (bb == 0.0) {
        MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        info->true_res = 0;
        return MGC_OK;
    }
    const double tol2 = p->tol * p->tol * bb;
    if (p->x_is_guess) {
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(residual(op, r, b, t, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
        info->true_res = std::sqrt(rr / bb);
        if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "FGCR: non-finite initial residual");
        if (rr <= tol2) return MGC_OK;
    } else {
        MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        MGC_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
    }
    int iters = 0;
    for (;;) {
        for (int j = 0; j < m && iters < p->max_iter; ++j) {
            double2 *wj = W->w[j], *zj = W->z[j];
            MGC_TRY(precondition(op, p, r, zj, s));
            MGC_TRY(apply_D64(op, zj, wj, s));
            // beta_i = <w_i, w_j>, four at a time
            for (int i0 = 0; i0 < j; i0 += 4) {
                const int cnt = (j - i0 < 4) ? j - i0 : 4;
                PtrList L{};
                for (int q = 0; q < cnt; ++q) L.p[q] = W->w[i0 + q];
                MGC_TRY(reduce<8>(
                    n,
                    [=] __device__(long long e, double *acc) {
                        const double2 v = wj[e];
#pragma unroll
                        for (int q = 0; q < 4; ++q)
                            if (q < cnt) acc_dot(acc + 2 * q, L.p[q][e], v);
                    },
                    W, sc + S_BETA + 2 * i0, s, cnt + 1));
            }
            // w_j -= sum beta_i w_i, z_j -= sum beta_i z_i; ||w_j||^2 and <w_j, r>
            PtrList Lw{}, Lz{};
            for (int q = 0; q < j; ++q) {
                Lw.p[q] = W->w[q];
                Lz.p[q] = W->z[q];
            }
            const double *beta = sc + S_BETA;
            MGC_TRY(reduce<3>(
                n,
                [=] __device__(long long e, double *acc) {
                    double2 wv = wj[e], zv = zj[e];
                    for (int q = 0; q < j; ++q) {
                        const double2 bq = ld2(beta + 2 * q);
                        wv = csub(wv, cmul(bq, Lw.p[q][e]));
                        zv = csub(zv, cmul(bq, Lz.p[q][e]));
                    }
                    wj[e] = wv;
                    zj[e] = zv;
                    acc_n2(acc, wv);
                    acc_dot(acc + 1, wv, r[e]);
                },
                W, sc + S_NW, s, 2 * j + 5));
            // normalise, then x += alpha z_j, r -= alpha w_j; ||r||^2 (1/||w_j|| and
            // alpha formed once, not per element)
            scalar_step([=] __device__() {
                const double inv = 1.0 / sqrt(sc[S_NW]);
                sc[S_ALPHA] = sc[S_WR] * inv;
                sc[S_ALPHA + 1] = sc[S_WR + 1] * inv;
                sc[S_OMEGA] = inv;
            }, s);
            MGC_TRY(reduce<1>(
                n,
                [=] __device__(long long e, double *acc) {
                    const double inv = sc[S_OMEGA];
                    const double2 alpha = ld2(sc + S_ALPHA);
                    double2 wv = wj[e], zv = zj[e];
                    wv = make_double2(wv.x * inv, wv.y * inv);
                    zv = make_double2(zv.x * inv, zv.y * inv);
                    wj[e] = wv;
                    zj[e] = zv;
                    x[e] = cadd(x[e], cmul(alpha, zv));
                    const double2 rv = csub(r[e], cmul(alpha, wv));
                    r[e] = rv;
                    acc_n2(acc, rv);
                },
                W, sc + S_RR, s, 8));
            ++iters;
            MGC_TRY(read_scalar(W, S_RR, &rr, s));
            MGC_TRY(check_device_status(op, s));
            if (bad(rr)) {
                info->iters = iters;
                info->true_res = NAN;
                return fail(MGC_ERR_BREAKDOWN, "FGCR: non-finite residual");
            }
            if (rr <= tol2) break;
        }
        // true residual
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(residual(op, r, b, t, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
        info->iters = iters;
        info->true_res = std::sqrt(rr / bb);
        if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "FGCR: non-finite true residual");
        if (rr <= tol2) return MGC_OK;
        if (iters >= p->max_iter) return MGC_NOT_CONVERGED;
        info->restarts++;
    }
}

// ------------------------------------------------------------------ flexible BiCGStab
// preconditioners for fbicgstab_impl: z = M v, returning a status
struct PreSAP {
    mgc_clover_s *op;
    const mgc_solve_params *p;
    cudaStream_t s;
    int operator()(const double2 *v, double2 *z) const { return precondition(op, p, v, z, s); }
};
static int mg_precondition(mgc_mg_s *M, const mgc_mg_params *mp, const double2 *v, double2 *z, cudaStream_t s);
struct PreMG {
    mgc_mg_s *M;
    const mgc_mg_params *mp;
    cudaStream_t s;
    int operator()(const double2 *v, double2 *z) const { return mg_precondition(M, mp, v, z, s); }
};

template <class PRE>
static int fbicgstab_impl(mgc_clover_s *op, const mgc_solve_params *p, mgc_solve_info *info, cudaStream_t s, PRE pre)
{
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    double2 *x = W->x, *r = W->r, *b = W->b, *t = W->t;
    double2 *r0 = W->w[0], *pv = W->w[1], *v = W->w[2], *sv = W->w[3];
    double2 *ph = W->z[0], *sh = W->z[1];
    double *sc = W->scal;
    double bb, rr;
    MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, b[e]); }, W, sc + S_BB, s, 1));
    MGC_TRY(read_scalar(W, S_BB, &bb, s));
    info->iters = 0;
    info->restarts = 0;
    if (bb == 0.0) {
        MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        info->true_res = 0;
        return MGC_OK;
    }
    if (!p->x_is_guess) MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
    const double tol2 = p->tol * p->tol * bb;
    int iters = 0;
    for (;;) {
        // r = b - D x, r0 = p = r, rho = <r0, r>
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(reduce<2>(
            n,
            [=] __device__(long long e, double *acc) {
                const double2 vv = csub(b[e], t[e]);
                r[e] = vv;
                r0[e] = vv;
                pv[e] = vv;
                acc_dot(acc, vv, vv);
            },
            W, sc + S_RHO, s, 5));
        if (iters == 0 && p->x_is_guess) {
            MGC_TRY(read_scalar(W, S_RHO, &rr, s));
            info->true_res = std::sqrt(rr / bb);
            if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "BiCGStab: non-finite initial residual");
            if (rr <= tol2) return MGC_OK;
        }
        bool restart = false;
        while (iters < p->max_iter) {
            MGC_TRY(pre(pv, ph));
            MGC_TRY(apply_D64(op, ph, v, s));
            MGC_TRY(reduce<2>(n, [=] __device__(long long e, double *acc) { acc_dot(acc, r0[e], v[e]); }, W, sc + S_R0V, s, 2));
            scalar_step([=] __device__() {
                const double2 a = cdiv(ld2(sc + S_RHO), ld2(sc + S_R0V));
                sc[S_ALPHA] = a.x;
                sc[S_ALPHA + 1] = a.y;
            }, s);
            // s = r - alpha v
            MGC_TRY(map(
                n,
                [=] __device__(long long e) { sv[e] = csub(r[e], cmul(ld2(sc + S_ALPHA), v[e])); },
                s, 3));
            MGC_TRY(pre(sv, sh));
            MGC_TRY(apply_D64(op, sh, t, s));
            MGC_TRY(reduce<3>(
                n,
                [=] __device__(long long e, double *acc) {
                    acc_dot(acc, t[e], sv[e]);
                    acc_n2(acc + 2, t[e]);
                },
                W, sc + S_TS, s, 2));
            scalar_step([=] __device__() {
                const double tt = sc[S_TT];
                sc[S_OMEGA] = tt > 0 ? sc[S_TS] / tt : 0.0;
                sc[S_OMEGA + 1] = tt > 0 ? sc[S_TS + 1] / tt : 0.0;
            }, s);
            // x += alpha ph + omega sh, r = s - omega t; ||r||^2 and <r0, r>
            MGC_TRY(reduce<3>(
                n,
                [=] __device__(long long e, double *acc) {
                    const double2 alpha = ld2(sc + S_ALPHA), omega = ld2(sc + S_OMEGA);
                    x[e] = cadd(x[e], cadd(cmul(alpha, ph[e]), cmul(omega, sh[e])));
                    const double2 rv = csub(sv[e], cmul(omega, t[e]));
                    r[e] = rv;
                    acc_n2(acc, rv);
                    acc_dot(acc + 1, r0[e], rv);
                },
                W, sc + S_RR, s, 8));
            ++iters;
            // slots S_RR, S_RR+1, S_RR+2 hold ||r||^2 and <r0, r>
            double h[3];
            MGC_CUDA(cudaMemcpyAsync(W->hscal, sc + S_RR, 3 * sizeof(double), cudaMemcpyDeviceToHost, s));
            MGC_CUDA(cudaStreamSynchronize(s));
            for (int k = 0; k < 3; ++k) h[k] = W->hscal[k];
            rr = h[0];
            if (bad(rr)) {
                info->iters = iters;
                info->true_res = NAN;
                return fail(MGC_ERR_BREAKDOWN, "BiCGStab: non-finite residual");
            }
            if (rr <= tol2) break;
            if (h[1] == 0.0 && h[2] == 0.0) { restart = true; break; }
            // p = r + beta (p - omega v), beta = (rho1 / rho)(alpha / omega); rho = rho1
            scalar_step([=] __device__() {
                const double2 beta = cmul(cdiv(ld2(sc + S_RR + 1), ld2(sc + S_RHO)),
                                          cdiv(ld2(sc + S_ALPHA), ld2(sc + S_OMEGA)));
                sc[S_BETAB] = beta.x;
                sc[S_BETAB + 1] = beta.y;
            }, s);
            MGC_TRY(map(
                n,
                [=] __device__(long long e) {
                    const double2 beta = ld2(sc + S_BETAB), omega = ld2(sc + S_OMEGA);
                    pv[e] = cadd(r[e], cmul(beta, csub(pv[e], cmul(omega, v[e]))));
                },
                s, 4));
            MGC_CUDA(cudaMemcpyAsync(sc + S_RHO, sc + S_RR + 1, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
        }
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(residual(op, r, b, t, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
        info->iters = iters;
        info->true_res = std::sqrt(rr / bb);
        if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "BiCGStab: non-finite true residual");
        if (rr <= tol2) return MGC_OK;
        if (iters >= p->max_iter) return MGC_NOT_CONVERGED;
        (void)restart;
        info->restarts++;
    }
}

static int fbicgstab(mgc_clover_s *op, const mgc_solve_params *p, mgc_solve_info *info, cudaStream_t s)
{
    return fbicgstab_impl(op, p, info, s, PreSAP{op, p, s});
}

// ------------------------------------------------------------------ multigrid solve (Sec. 3)
// flexible BiCGStab with FP64 vectors and operator, preconditioned by the
// two-level preconditioner (FP32 inside; it takes v / ||v||)
static int mg_precondition(mgc_mg_s *M, const mgc_mg_params *mp, const double2 *v, double2 *z, cudaStream_t s)
{
    mgc_clover_s *op = mg_operator(M);
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, v[e]); }, W, W->scal + S_NW, s, 1));
    double nn = 0.0;
    MGC_TRY(read_scalar(W, S_NW, &nn, s));
    if (bad(nn)) return fail(MGC_ERR_BREAKDOWN, "multigrid: non-finite vector");
    return mg_precond64(M, mp, v, z, std::sqrt(nn), s);
}

int mg_solve(mgc_mg_s *M, const double *b, double *x, const mgc_solve_params *p, const mgc_mg_params *mp,
             mgc_solve_info *info, cudaStream_t s)
{
    mgc_clover_s *op = mg_operator(M);
    if (!(p->tol > 0) || p->max_iter < 1) return fail(MGC_ERR_INVALID_ARG, "tol or max_iter out of range");
    MGC_TRY(ensure_work(op, 1, 4, 64));
    SolverWork *W = op->work;
    const Geom &g = op->gauge->lat->g;
    const size_t vb = spinor_bytes(g, 64, 1);
    if (p->on_device) {
        MGC_TRY(launch_pack(g, 64, 1, b, W->b, s));
        if (p->x_is_guess) MGC_TRY(launch_pack(g, 64, 1, x, W->x, s));
    } else {
        MGC_CUDA(cudaMemcpyAsync(W->stage, b, vb, cudaMemcpyHostToDevice, s));
        MGC_TRY(launch_pack(g, 64, 1, (const double *)W->stage, W->b, s));
        if (p->x_is_guess) {
            MGC_CUDA(cudaMemcpyAsync(W->stage, x, vb, cudaMemcpyHostToDevice, s));
            MGC_TRY(launch_pack(g, 64, 1, (const double *)W->stage, W->x, s));
        }
    }
    *info = mgc_solve_info{MGC_OK, 0, 0, 0.0};
    const int st = fbicgstab_impl(op, p, info, s, PreMG{M, mp, s});
    info->status = st;
    if (st != MGC_OK && st != MGC_NOT_CONVERGED) return st;
    if (p->on_device) {
        MGC_TRY(launch_unpack(g, 64, 1, W->x, x, s));
    } else {
        MGC_TRY(launch_unpack(g, 64, 1, W->x, (double *)W->stage, s));
        MGC_CUDA(cudaMemcpyAsync(x, W->stage, vb, cudaMemcpyDeviceToHost, s));
    }
    MGC_CUDA(cudaStreamSynchronize(s));
    MGC_TRY(check_device_status(op, s));
    return st;
}

// ------------------------------------------------------------------ two-level solve
// FP64 defect correction (the double-precision Richardson iteration around a
// single-precision solver of Sec. 2) with an FP32 inner FGCR(m) preconditioned
// by SAP:  r = b - D x in FP64;  solve D e = r to inner_tol ||r|| with FP32
// vectors and the FP32 operator (r enters as its FP32 copy times a power of
// two 2^k, see unit_exp); x += 2^-k e in FP64;  repeat until the FP64 true
// residual meets tol.  Inner
// products of the FP32 vectors accumulate in FP32 over chunks of entries per
// thread and in FP64 beyond that; the Gram-Schmidt coefficients and step
// lengths are FP64 host scalars.  The inner
// FGCR never rescales or orthogonalises the z vectors: with w'_j = w_j -
// sum_i c_ij w'_i and alpha_j = <w'_j, r>/||w'_j||^2, the correction is
// e = sum_j gamma_j z_j with R gamma = alpha, R unit upper triangular with
// R_ij = c_ij, applied once per inner solve.


template <int NV>
__device__ __forceinline__ void finish_reduce(double *acc, double (*sh)[RT / 32], bool *last, double *partial,
                                              unsigned *counter, double *out)
{
    block_reduce<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[blockIdx.x * NV + k] = acc[k];
        __threadfence();
        *last = (atomicAdd(counter, 1u) == gridDim.x - 1);
    }
    __syncthreads();
    if (!*last) return;
    __threadfence();
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0;
    for (int bi = threadIdx.x; bi < (int)gridDim.x; bi += RT)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += __ldcg(partial + bi * NV + k);
    block_reduce<NV>(acc, sh);
    if (threadIdx.x == 0) {
#pragma unroll
        for (int k = 0; k < NV; ++k) out[k] = acc[k];
        *counter = 0;
    }
}

// FP32 vectors are read as float4 (two complex entries per load).  Each thread
// takes U4 independent float4 entries per step (grid stride apart, so a warp's
// loads stay contiguous) to keep enough loads in flight to cover HBM latency;
// its FP32 partial sums go to FP64 every flush_steps<NV>() steps.  With
// several sums (the Gram-Schmidt inner products) a flush per step made the
// kernel FP64-bound on GB300 (NV conversions and additions per four entries),
// so those flush every fourth step: an FP32 partial then holds 16 float4
// entries.
constexpr int U4 = 4;
template <int NV>
__host__ __device__ constexpr int flush_steps() { return NV >= 2 ? 4 : 1; }

template <int NV, class F>
__global__ void __launch_bounds__(RT) k_reduce32(long long n4, F f, double *partial, unsigned *counter, double *out)
{
    static_assert(NV <= PART_NV, "more accumulators than the partial-sum area holds");
    __shared__ double sh[NV][RT / 32];
    __shared__ bool last;
    double acc[NV];
    float facc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) {
        acc[k] = 0;
        facc[k] = 0.f;
    }
    const long long stride = (long long)gridDim.x * RT;
    long long e = (long long)blockIdx.x * RT + threadIdx.x;
    int step = 0;
    for (; e + (U4 - 1) * stride < n4; e += U4 * stride) {
#pragma unroll
        for (int u = 0; u < U4; ++u) f(e + u * stride, facc);
        if (++step == flush_steps<NV>()) {
            step = 0;
#pragma unroll
            for (int k = 0; k < NV; ++k) {
                acc[k] += (double)facc[k];
                facc[k] = 0.f;
            }
        }
    }
    for (; e < n4; e += stride) f(e, facc);
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] += (double)facc[k];
    finish_reduce<NV>(acc, sh, &last, partial, counter, out);
}

template <class F>
__global__ void __launch_bounds__(RT) k_map32(long long n4, F f)
{
    const long long stride = (long long)gridDim.x * RT;
    long long e = (long long)blockIdx.x * RT + threadIdx.x;
    for (; e + (U4 - 1) * stride < n4; e += U4 * stride)
#pragma unroll
        for (int u = 0; u < U4; ++u) f(e + u * stride);
    for (; e < n4; e += stride) f(e);
}

// blocks for the FP32 vector kernels: every block resident at once (a whole
// number of waves over the SMs), within the partial-sum area
template <class K>
static int grid32(K kern, long long n4)
{
    // per device (SM counts may differ), per kernel instantiation
    static int cached[64] = {};
    int dev = 0;
    cudaGetDevice(&dev);
    int &c = cached[dev >= 0 && dev < 64 ? dev : 0];
    if (!c) {
        int sms = 0, per = 0;
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, RT, 0);
        if (sms < 1) sms = 1;
        if (per < 1) per = 1;
        while (per > 1 && sms * per > RGRID_MAX) --per;
        c = sms * per > RGRID_MAX ? RGRID_MAX : sms * per;
    }
    long long need = (n4 + (long long)RT * U4 - 1) / ((long long)RT * U4);
    if (need < 1) need = 1;
    return need < c ? (int)need : c;
}

// n: complex entries (even); f takes a float4 index
template <int NV, class F>
static int reduce32(long long n, F f, SolverWork *W, double *out, cudaStream_t s, double bytes)
{
    const long long n4 = n / 2;
    auto kern = k_reduce32<NV, F>;
    kern<<<grid32(kern, n4), RT, 0, s>>>(n4, f, W->partial, W->counter, out);
    MGC_CUDA(cudaGetLastError());
    count(1, bytes);
    return MGC_OK;
}

template <class F>
static int map32(long long n, F f, cudaStream_t s, double bytes)
{
    const long long n4 = n / 2;
    auto kern = k_map32<F>;
    kern<<<grid32(kern, n4), RT, 0, s>>>(n4, f);
    MGC_CUDA(cudaGetLastError());
    count(1, bytes);
    return MGC_OK;
}

__device__ __forceinline__ void facc_dot(float *acc, float2 a, float2 b)
{
    acc[0] = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[0]));
    acc[1] = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc[1]));
}
__device__ __forceinline__ void facc_n2(float *acc, float2 a) { acc[0] = fmaf(a.x, a.x, fmaf(a.y, a.y, acc[0])); }
__device__ __forceinline__ float2 lo2(float4 v) { return make_float2(v.x, v.y); }
__device__ __forceinline__ float2 hi2(float4 v) { return make_float2(v.z, v.w); }
// v -= c u for the two complex entries of a float4
__device__ __forceinline__ void csub4(float4 &v, float2 c, float4 u)
{
    v.x -= c.x * u.x - c.y * u.y;
    v.y -= c.x * u.y + c.y * u.x;
    v.z -= c.x * u.z - c.y * u.w;
    v.w -= c.x * u.w + c.y * u.z;
}

struct PtrList32 {
    const float2 *p[MAXM];
};
struct PtrList4 {
    const float4 *p[MAXM];
};
struct CoefList {
    float2 c[MAXM];
};

// read nd doubles of the scalar area (synchronises)
static int read_scalars(SolverWork *W, int slot, int nd, double *out, cudaStream_t s)
{
    MGC_CUDA(cudaMemcpyAsync(W->hscal, W->scal + slot, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nd; ++k) out[k] = W->hscal[k];
    return MGC_OK;
}

// z = M v for FP32 v, z
static int precondition32(mgc_clover_s *op, const mgc_solve_params *p, const float2 *v, float2 *z, cudaStream_t s)
{
    const Geom &g = op->gauge->lat->g;
    SolverWork *W = op->work;
    if (p->precond == 0) {
        MGC_CUDA(cudaMemcpyAsync(z, v, spinor_bytes(g, 32, 1), cudaMemcpyDeviceToDevice, s));
        return MGC_OK;
    }
    if (p->smoother_prec == 32) {
        MGC_CUDA(cudaMemsetAsync(z, 0, spinor_bytes(g, 32, 1), s));
        return run_sap(op, p, 32, v, z, s);
    }
    MGC_TRY(launch_convert(g, 1, 32, v, 16, W->rl, s));
    MGC_CUDA(cudaMemsetAsync(W->zl, 0, spinor_bytes(g, 16, 1), s));
    MGC_TRY(run_sap(op, p, 16, W->rl, W->zl, s));
    return launch_convert(g, 1, 16, W->zl, 32, z, s);
}

typedef std::complex<double> zd;

// an FP16 packed spinor of one right-hand side: data, then one scale per site
static Spinor16 view16(const Geom &g, void *p)
{
    uint4 *d = (uint4 *)p;
    return Spinor16{d, (float *)(d + (size_t)g.V * 3), g.lvb};
}

// the FP16-smoother path of the inner FGCR: the smoother's FP16 output z_j is
// kept as it is (no FP32 copy), the FP32 operator reads it directly, and the
// residual update also writes the FP16 residual the smoother reads
static bool fp16_directions(const mgc_solve_params *p) { return p->precond != 0 && p->smoother_prec == 16; }

// One pass over sites for the FP16-smoother path: w'_j = w_j - sum_i c_i w'_i
// and r -= alpha w'_j on the FP32 vectors, the FP16 copy of the new r, and
// ||w'_j||^2, ||r||^2 into two device scalars from slot on
static int orth_update_sites(mgc_clover_s *op, float2 *wj, const PtrList4 &Lw, const CoefList &C, int j, float2 alpha,
                             float2 *r, void *rl, int slot, cudaStream_t s)
{
    SolverWork *W = op->work;
    const Geom g = op->gauge->lat->g;
    const int lvb = g.lvb;
    const Spinor32 Wj{(float4 *)wj, lvb}, R{(float4 *)r, lvb};
    const Spinor16 RL = view16(g, rl);
    auto f = [=] __device__(long long i, double *acc) {
        Cx<float> v[12];
        Wj.load((int)i, v);
#pragma unroll
        for (int q = 0; q < MAXM; ++q)
            if (q < j) {
                const Spinor32 Wq{const_cast<float4 *>(Lw.p[q]), lvb};
                Cx<float> u[12];
                Wq.load((int)i, u);
                const Cx<float> c = {C.c[q].x, C.c[q].y};
#pragma unroll
                for (int k = 0; k < 12; ++k) v[k] = v[k] - c * u[k];
            }
        Wj.store((int)i, v);
        Cx<float> rv[12];
        R.load((int)i, rv);
        const Cx<float> a = {alpha.x, alpha.y};
        float nw = 0.f, nr = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            nw += norm2(v[k]);
            rv[k] = rv[k] - a * v[k];
            nr += norm2(rv[k]);
        }
        R.store((int)i, rv);
        RL.store((int)i, rv);
        acc[0] += nw;
        acc[1] += nr;
    };
    k_reduce<2><<<red_grid(g.V), RT, 0, s>>>((long long)g.V, f, W->partial, W->counter, W->scal + slot);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (96.0 * (j + 4) + 52.0));
    return MGC_OK;
}

// <L_q, v> for the CNT vectors of L (2 CNT sums) and, when norm is set,
// ||v||^2 (one more), into 2 CNT + 1 device scalars from out on; one
// instantiation per count, so only the sums in use are carried to FP64
template <int CNT>
static int multidot(long long n, const PtrList4 &L, const float4 *v, bool norm, SolverWork *W, double *out,
                    cudaStream_t s)
{
    return reduce32<2 * CNT + 1>(
        n,
        [=] __device__(long long e, float *acc) {
            const float4 x = v[e];
#pragma unroll
            for (int q = 0; q < CNT; ++q) {
                const float4 a = L.p[q][e];
                facc_dot(acc + 2 * q, lo2(a), lo2(x));
                facc_dot(acc + 2 * q, hi2(a), hi2(x));
            }
            if (norm) {
                facc_n2(acc + 2 * CNT, lo2(x));
                facc_n2(acc + 2 * CNT, hi2(x));
            }
        },
        W, out, s, 8.0 * n * (CNT + 1));
}

// inner FGCR on W->r32 (||r||^2 = rr0 on entry, the residual on exit; with
// the FP16 smoother W->rl holds the FP16 copy of r on entry and is kept
// current); stops at ||r|| <= tol_in sqrt(rr0); fills gamma for the k
// directions it built; *rr_out = final ||r||^2
static int inner_fgcr32(mgc_clover_s *op, const mgc_solve_params *p, double tol_in, double rr0, int max_it,
                        int *k_out, std::vector<zd> &gamma, double *rr_out, cudaStream_t s)
{
    SolverWork *W = op->work;
    const Geom &gm = op->gauge->lat->g;
    const long long n = (long long)gm.V * 12;
    const bool h16 = fp16_directions(p);  // W->rl holds the FP16 copy of r on entry
    const int m = p->restart < max_it ? p->restart : max_it;
    float2 *r = W->r32;
    double *sc = W->scal;
    std::vector<double> n2(m);
    std::vector<zd> alpha(m);
    std::vector<std::vector<zd>> R(m, std::vector<zd>(m, zd(0, 0)));
    double rr = rr0;
    int k = 0;
    for (int j = 0; j < m; ++j) {
        float2 *zj = W->z32[j], *wj = W->w32[j];
        if (h16) {
            MGC_CUDA(cudaMemsetAsync(W->z16[j], 0, spinor_bytes(gm, 16, 1), s));
            MGC_TRY(run_sap(op, p, 16, W->rl, W->z16[j], s));
            MGC_TRY(launch_dirac_from16(op, W->z16[j], wj, s));
        } else {
            MGC_TRY(precondition32(op, p, r, zj, s));
            MGC_TRY(launch_dirac(op, 32, false, zj, wj, 1, s));
        }
        // d_i = <w'_i, w_j> (i < j) and rho = <w_j, r>, eight at a time, and
        // ||w_j||^2 with the first eight
        std::vector<zd> d(j + 1);
        double ww = 0.0;
        for (int i0 = 0; i0 <= j; i0 += 8) {
            const int cnt = (j + 1 - i0 < 8) ? j + 1 - i0 : 8;
            const bool first = i0 == 0;
            // <L_q, w_j> with L = (w'_0 .. w'_{j-1}, r)
            PtrList4 L{};
            for (int q = 0; q < cnt; ++q) L.p[q] = (const float4 *)((i0 + q < j) ? W->w32[i0 + q] : r);
            switch (cnt) {
                case 1: MGC_TRY(multidot<1>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                case 2: MGC_TRY(multidot<2>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                case 3: MGC_TRY(multidot<3>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                case 4: MGC_TRY(multidot<4>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                case 5: MGC_TRY(multidot<5>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                case 6: MGC_TRY(multidot<6>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                case 7: MGC_TRY(multidot<7>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
                default: MGC_TRY(multidot<8>(n, L, (const float4 *)wj, first, W, sc + S_BETA, s)); break;
            }
            double h[17];
            MGC_TRY(read_scalars(W, S_BETA, 2 * cnt + 1, h, s));
            for (int q = 0; q < cnt; ++q) d[i0 + q] = zd(h[2 * q], h[2 * q + 1]);
            if (first) ww = h[2 * cnt];
        }
        const zd rho = std::conj(d[j]);  // <w_j, r>
        // w'_j = w_j - sum_i c_i w'_i, c_i = d_i / ||w'_i||^2
        CoefList C{};
        PtrList4 Lw{};
        double nw_est = ww;  // ||w'_j||^2 = ||w_j||^2 - sum_i |d_i|^2 / ||w'_i||^2 (w'_i orthogonal)
        for (int i = 0; i < j; ++i) {
            const zd c = d[i] / n2[i];
            R[i][j] = c;
            C.c[i] = make_float2((float)c.real(), (float)c.imag());
            Lw.p[i] = (const float4 *)W->w32[i];
            nw_est -= std::norm(d[i]) / n2[i];
        }
        float4 *wj4 = (float4 *)wj;
        float4 *r4 = (float4 *)r;
        if (!bad(ww) && nw_est > 1e-3 * ww) {
            // one pass: orthogonalise w_j and update r with alpha from the
            // estimate; the exact ||w'_j||^2 (for later coefficients) and
            // ||r||^2 come back from the same pass
            alpha[j] = rho / nw_est;
            const float2 a = make_float2((float)alpha[j].real(), (float)alpha[j].imag());
            if (h16) {
                MGC_TRY(orth_update_sites(op, wj, Lw, C, j, a, r, W->rl, S_BETA, s));
            } else {
                MGC_TRY(reduce32<2>(
                n,
                [=] __device__(long long e, float *acc) {
                    float4 v = wj4[e];
#pragma unroll
                    for (int i = 0; i < MAXM; ++i)
                        if (i < j) csub4(v, C.c[i], Lw.p[i][e]);
                    wj4[e] = v;
                    facc_n2(acc, lo2(v));
                    facc_n2(acc, hi2(v));
                    float4 u = r4[e];
                    csub4(u, a, v);
                    r4[e] = u;
                    facc_n2(acc + 1, lo2(u));
                    facc_n2(acc + 1, hi2(u));
                },
                W, sc + S_BETA, s, 8.0 * n * (j + 4)));
            }
            double h2[2];
            MGC_TRY(read_scalars(W, S_BETA, 2, h2, s));
            if (bad(h2[0]) || h2[0] == 0.0) return fail(MGC_ERR_BREAKDOWN, "inner FGCR: zero or non-finite direction");
            n2[j] = h2[0];
            rr = h2[1];
            k = j + 1;
            if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "inner FGCR: non-finite residual");
            if (rr <= tol_in * tol_in * rr0) break;
            continue;
        }
        // strong cancellation in the estimate: orthogonalise, then update r
        MGC_TRY(reduce32<1>(
            n,
            [=] __device__(long long e, float *acc) {
                float4 v = wj4[e];
#pragma unroll
                for (int i = 0; i < MAXM; ++i)
                    if (i < j) csub4(v, C.c[i], Lw.p[i][e]);
                wj4[e] = v;
                facc_n2(acc, lo2(v));
                facc_n2(acc, hi2(v));
            },
            W, sc + S_NW, s, 8.0 * n * (j + 2)));
        double nw;
        MGC_TRY(read_scalars(W, S_NW, 1, &nw, s));
        if (bad(nw) || nw == 0.0) return fail(MGC_ERR_BREAKDOWN, "inner FGCR: zero or non-finite direction");
        n2[j] = nw;
        alpha[j] = rho / nw;
        const float2 a = make_float2((float)alpha[j].real(), (float)alpha[j].imag());
        MGC_TRY(reduce32<1>(
            n,
            [=] __device__(long long e, float *acc) {
                float4 v = r4[e];
                csub4(v, a, wj4[e]);
                r4[e] = v;
                facc_n2(acc, lo2(v));
                facc_n2(acc, hi2(v));
            },
            W, sc + S_RR, s, 8.0 * n * 3));
        if (h16) MGC_TRY(launch_convert(gm, 1, 32, r, 16, W->rl, s));
        MGC_TRY(read_scalars(W, S_RR, 1, &rr, s));
        k = j + 1;
        if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "inner FGCR: non-finite residual");
        if (rr <= tol_in * tol_in * rr0) break;
    }
    gamma.assign(k, zd(0, 0));
    for (int i = k - 1; i >= 0; --i) {
        zd g = alpha[i];
        for (int j = i + 1; j < k; ++j) g -= R[i][j] * gamma[j];
        gamma[i] = g;
    }
    *k_out = k;
    *rr_out = rr;
    return MGC_OK;
}

// r32 = scale (b - t) site by site (the FP64 and FP32 packed layouts differ;
// t may be null: r32 = scale b), its FP16 copy into rl when rl is given (the
// FP16 smoother's input), and the unscaled ||b - t||^2 into a device scalar
// slot.  The FP64 residual itself is not kept: the inner solve only needs its
// FP32 copy.
static int residual_to32(mgc_clover_s *op, const double2 *b, const double2 *t, float2 *r32, void *rl, double scale,
                         int slot, cudaStream_t s)
{
    // scale (a power of two) is applied after the conversion to FP32, where
    // the product is exact and costs no FP64 instruction, unless it is so far
    // from 1 that the unscaled values could leave FP32's range
    const bool wide = scale > 0x1p90 || scale < 0x1p-90;
    const float sf = wide ? 1.0f : (float)scale;  // (float) only of a value in FP32's range
    SolverWork *W = op->work;
    const Geom g = op->gauge->lat->g;
    const Spinor64 B{const_cast<double2 *>(b), g.lvb}, T{const_cast<double2 *>(t), g.lvb};
    const Spinor32 R{reinterpret_cast<float4 *>(r32), g.lvb};
    const bool has_t = t != nullptr, has_l = rl != nullptr;
    const Spinor16 RL = has_l ? view16(g, rl) : Spinor16{nullptr, nullptr, g.lvb};
    auto f = [=] __device__(long long i, double *acc) {
        Cx<double> v[12];
        Cx<float> w[12];
        B.load((int)i, v);
        if (has_t) {
            Cx<double> u[12];
            T.load((int)i, u);
#pragma unroll
            for (int k = 0; k < 12; ++k) v[k] = v[k] - u[k];
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[0] = fma(v[k].r, v[k].r, fma(v[k].i, v[k].i, acc[0]));
        if (wide) {
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] = Cx<float>{(float)(scale * v[k].r), (float)(scale * v[k].i)};
        } else {
#pragma unroll
            for (int k = 0; k < 12; ++k) w[k] = Cx<float>{(float)v[k].r * sf, (float)v[k].i * sf};
        }
        R.store((int)i, w);
        if (has_l) RL.store((int)i, w);
    };
    k_reduce<1><<<red_grid(g.V), RT, 0, s>>>((long long)g.V, f, W->partial, W->counter, W->scal + slot);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * ((has_t ? 2 : 1) * 192.0 + 96.0 + (has_l ? 52.0 : 0.0)));
    return MGC_OK;
}

// x += es sum_j gamma_j z_j site by site: the sum in FP32 (its rounding is far
// below the inner tolerance), the update of x in FP64
static int axpy_sum32(mgc_clover_s *op, double2 *x, const PtrList4 &Lz, const CoefList &G, int k, double es,
                      cudaStream_t s)
{
    const Geom g = op->gauge->lat->g;
    const Spinor64 X{x, g.lvb};
    const int lvb = g.lvb;
    auto f = [=] __device__(long long i) {
        Cx<float> e[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) e[c] = Cx<float>{0.f, 0.f};
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < k) {
                const Spinor32 Z{const_cast<float4 *>(Lz.p[j]), lvb};
                Cx<float> z[12];
                Z.load((int)i, z);
                const Cx<float> gj = {G.c[j].x, G.c[j].y};
#pragma unroll
                for (int c = 0; c < 12; ++c) e[c] = cfma(gj, z[c], e[c]);
            }
        Cx<double> v[12];
        X.load((int)i, v);
#pragma unroll
        for (int c = 0; c < 12; ++c) v[c] = Cx<double>{fma(es, (double)e[c].r, v[c].r), fma(es, (double)e[c].i, v[c].i)};
        X.store((int)i, v);
    };
    k_map<<<red_grid(g.V), RT, 0, s>>>((long long)g.V, f);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (2 * 192.0 + 96.0 * k));
    return MGC_OK;
}

// x += es sum_j gamma_j z_j for FP16 z_j (the FP16-smoother path), as axpy_sum32
struct Spinor16List {
    Spinor16 z[MAXM];
};
static int axpy_sum16(mgc_clover_s *op, double2 *x, const Spinor16List &Z, const CoefList &G, int k, double es,
                      cudaStream_t s)
{
    const Geom g = op->gauge->lat->g;
    const Spinor64 X{x, g.lvb};
    auto f = [=] __device__(long long i) {
        Cx<float> e[12];
#pragma unroll
        for (int c = 0; c < 12; ++c) e[c] = Cx<float>{0.f, 0.f};
#pragma unroll
        for (int j = 0; j < MAXM; ++j)
            if (j < k) {
                Cx<float> z[12];
                Z.z[j].load((int)i, z);
                const Cx<float> gj = {G.c[j].x, G.c[j].y};
#pragma unroll
                for (int c = 0; c < 12; ++c) e[c] = cfma(gj, z[c], e[c]);
            }
        Cx<double> v[12];
        X.load((int)i, v);
#pragma unroll
        for (int c = 0; c < 12; ++c) v[c] = Cx<double>{fma(es, (double)e[c].r, v[c].r), fma(es, (double)e[c].i, v[c].i)};
        X.store((int)i, v);
    };
    k_map<<<red_grid(g.V), RT, 0, s>>>((long long)g.V, f);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (2 * 192.0 + 52.0 * k));
    return MGC_OK;
}

// The exponent of the power of two nearest 1 / (the rms of the 2n real
// components of a vector whose squared norm is rr): the inner solve works on
// the residual times 2^e.  Scaling by a power of two is exact and commutes
// with every rounding, so the inner solve's results are those of the
// unscaled residual wherever that stays in FP32's normal range, and it keeps
// FP32's sums of squares in range for any residual whose squared norm is a
// normal FP64 number.  Scaled norms are formed with ldexp, never by
// multiplying with 2^e twice (which would overflow for the smallest ones).
static int unit_exp(double rr, long long n)
{
    if (!(rr > 0.0) || !std::isfinite(rr)) return 0;
    int e = 0;
    std::frexp(std::sqrt(rr / (2.0 * (double)n)), &e);
    return -e;
}

static int two_level(mgc_clover_s *op, const mgc_solve_params *p, mgc_solve_info *info, cudaStream_t s)
{
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    double2 *x = W->x, *b = W->b, *t = W->t;
    float2 *r32 = W->r32;
    void *rl = fp16_directions(p) ? W->rl : nullptr;  // the FP16 smoother's input
    double *sc = W->scal;
    double bb, rr;
    int re = 0;  // r32 (and its FP16 copy) = 2^re (b - D x)
    info->iters = 0;
    info->restarts = 0;
    info->true_res = 0;
    if (p->x_is_guess) {
        MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, b[e]); }, W, sc + S_BB, s, 1));
        MGC_TRY(read_scalar(W, S_BB, &bb, s));
        if (bb == 0.0) {
            MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
            return MGC_OK;
        }
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(residual_to32(op, b, t, r32, rl, 1.0, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
    } else {
        // x = 0: r = b, and ||b||^2 from the same pass
        MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        MGC_TRY(residual_to32(op, b, nullptr, r32, rl, 1.0, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
        bb = rr;
        if (bb == 0.0) return MGC_OK;
    }
    // a first residual far from unit rms (beyond 2^+-30) is written again at
    // its unit scale; later ones are written at the unit scale of the inner
    // solve's final residual, the prediction of theirs
    if (std::isfinite(rr) && rr > 0.0) {
        const int e = unit_exp(rr, n);
        if (e > 30 || e < -30) {
            re = e;
            MGC_TRY(residual_to32(op, b, p->x_is_guess ? t : nullptr, r32, rl, std::ldexp(1.0, re), S_RR, s));
        }
    }
    const double tol2 = p->tol * p->tol * bb;
    int iters = 0;
    for (;;) {
        info->true_res = std::sqrt(rr / bb);
        if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "defect correction: non-finite residual");
        if (rr <= tol2) return MGC_OK;
        if (iters >= p->max_iter) return MGC_NOT_CONVERGED;
        // the last pass only needs to reach tol ||b||
        double tin = p->inner_tol;
        const double need = 0.5 * p->tol * std::sqrt(bb / rr);
        if (need > tin) tin = need;
        int k = 0;
        double rri;
        std::vector<zd> gamma;
        MGC_TRY(inner_fgcr32(op, p, tin, std::ldexp(rr, 2 * re), p->max_iter - iters, &k, gamma, &rri, s));
        iters += k;
        // x += e, e = sum_j gamma_j z_j
        CoefList G{};
        for (int j = 0; j < k; ++j) G.c[j] = make_float2((float)gamma[j].real(), (float)gamma[j].imag());
        if (rl) {
            Spinor16List Z{};
            for (int j = 0; j < k; ++j) Z.z[j] = view16(op->gauge->lat->g, W->z16[j]);
            MGC_TRY(axpy_sum16(op, x, Z, G, k, std::ldexp(1.0, -re), s));
        } else {
            PtrList4 Lz{};
            for (int j = 0; j < k; ++j) Lz.p[j] = (const float4 *)W->z32[j];
            MGC_TRY(axpy_sum32(op, x, Lz, G, k, std::ldexp(1.0, -re), s));
        }
        // the inner solve predicts that this x meets the tolerance: it goes to
        // the host (host-pointer solves) while the FP64 residual checks it
        if (W->host_x && std::ldexp(rri, -2 * re) <= tol2) MGC_TRY(copy_x_early(op, s));
        MGC_TRY(apply_D64(op, x, t, s));
        if (rri > 0.0 && std::isfinite(rri)) re = unit_exp(std::ldexp(rri, -2 * re), n);
        MGC_TRY(residual_to32(op, b, t, r32, rl, std::ldexp(1.0, re), S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
        if (!(rr <= tol2)) MGC_TRY(join_copy(W, s));  // x changes again
        info->iters = iters;
        info->restarts++;
        MGC_TRY(check_device_status(op, s));
    }
}

// ------------------------------------------------------------------ QWS solve
// The paper's QWS solver (Sec. 2) for D x = b.  A = C^-1 D; the source of the
// A-system is C^-1 r.  FP64 Richardson: r = b - D x (FP64), stop when
// ||r|| <= tol ||b||; otherwise r_A = C^-1 r (FP64), solve (A M) y = r_A/||r_A||
// with an FP32 BiCGStab to the inner tolerance, where M is the multiplicative
// SAP for A with n_mr Jacobi iterations per domain (a fixed linear operator, so
// plain BiCGStab applies) and A the FP32 operator; then x += ||r_A|| M y in
// FP64.  BiCGStab scalars are FP64 host values; its inner products accumulate
// as in the two-level solve.

// z = M v for FP32 v, z (the SAP for A at the smoother precision)
static int precondition32_A(mgc_clover_s *op, const mgc_solve_params *p, const float2 *v, float2 *z, cudaStream_t s)
{
    const Geom &g = op->gauge->lat->g;
    SolverWork *W = op->work;
    if (p->smoother_prec == 32) {
        MGC_CUDA(cudaMemsetAsync(z, 0, spinor_bytes(g, 32, 1), s));
        return launch_sap_A(op, 32, v, z, 1, p->n_cy, p->n_mr, 1, s);
    }
    MGC_TRY(launch_convert(g, 1, 32, v, 16, W->rl, s));
    MGC_CUDA(cudaMemsetAsync(W->zl, 0, spinor_bytes(g, 16, 1), s));
    MGC_TRY(launch_sap_A(op, 16, W->rl, W->zl, 1, p->n_cy, p->n_mr, 1, s));
    return launch_convert(g, 1, 16, W->zl, 32, z, s);
}

// out = A M v (tmp receives M v)
static int apply_AM(mgc_clover_s *op, const mgc_solve_params *p, const float2 *v, float2 *tmp, float2 *out,
                    cudaStream_t s)
{
    MGC_TRY(precondition32_A(op, p, v, tmp, s));
    return launch_apply_A(op, 32, tmp, out, 1, s);
}

__device__ __forceinline__ void facc_cdot(float *acc, float4 a, float4 b)
{
    facc_dot(acc, lo2(a), lo2(b));
    facc_dot(acc, hi2(a), hi2(b));
}

// BiCGStab on (A M) y = r32 (unit norm) from y = 0 to ||residual|| <= tin;
// y is left in W->z32[2]; *k_out counts iterations
static int inner_bicgstab32(mgc_clover_s *op, const mgc_solve_params *p, double tin, int max_it, int *k_out,
                            cudaStream_t s)
{
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    double *sc = W->scal;
    float4 *rr = (float4 *)W->w32[0], *r0 = (float4 *)W->w32[1], *pv = (float4 *)W->w32[2];
    float4 *v = (float4 *)W->w32[3], *sv = (float4 *)W->z32[0], *tv = (float4 *)W->z32[1];
    float4 *y = (float4 *)W->z32[2];
    float2 *tmp = W->z32[3];
    const size_t vb = spinor_bytes(op->gauge->lat->g, 32, 1);
    MGC_CUDA(cudaMemcpyAsync(rr, W->r32, vb, cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemcpyAsync(r0, W->r32, vb, cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemcpyAsync(pv, W->r32, vb, cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemsetAsync(y, 0, vb, s));
    double h[4];
    MGC_TRY(reduce32<2>(n, [=] __device__(long long e, float *acc) { facc_cdot(acc, r0[e], rr[e]); }, W, sc + S_RHO, s,
                        8.0 * n * 2));
    MGC_TRY(read_scalars(W, S_RHO, 2, h, s));
    zd rho(h[0], h[1]);
    int k = 0;
    while (k < max_it) {
        MGC_TRY(apply_AM(op, p, (const float2 *)pv, tmp, (float2 *)v, s));
        MGC_TRY(reduce32<2>(n, [=] __device__(long long e, float *acc) { facc_cdot(acc, r0[e], v[e]); }, W,
                            sc + S_R0V, s, 8.0 * n * 2));
        MGC_TRY(read_scalars(W, S_R0V, 2, h, s));
        const zd r0v(h[0], h[1]);
        if (bad(std::abs(r0v)) || r0v == zd(0, 0)) return fail(MGC_ERR_BREAKDOWN, "QWS BiCGStab: <r0, v> = 0");
        const zd alpha = rho / r0v;
        const float2 a = make_float2((float)alpha.real(), (float)alpha.imag());
        MGC_TRY(map32(
            n,
            [=] __device__(long long e) {
                float4 t4 = rr[e];
                csub4(t4, a, v[e]);
                sv[e] = t4;
            },
            s, 8.0 * n * 3));
        MGC_TRY(apply_AM(op, p, (const float2 *)sv, tmp, (float2 *)tv, s));
        MGC_TRY(reduce32<3>(
            n,
            [=] __device__(long long e, float *acc) {
                const float4 t4 = tv[e];
                facc_n2(acc, lo2(t4));
                facc_n2(acc, hi2(t4));
                facc_cdot(acc + 1, t4, sv[e]);
            },
            W, sc + S_TS, s, 8.0 * n * 2));
        MGC_TRY(read_scalars(W, S_TS, 3, h, s));
        const double tt = h[0];
        const zd omega = tt > 0 ? zd(h[1], h[2]) / tt : zd(0, 0);
        const float2 w = make_float2((float)omega.real(), (float)omega.imag());
        // y += alpha p + omega s; r = s - omega t; ||r||^2 and <r0, r>
        MGC_TRY(reduce32<3>(
            n,
            [=] __device__(long long e, float *acc) {
                float4 yy = y[e];
                const float4 s4 = sv[e];
                csub4(yy, make_float2(-a.x, -a.y), pv[e]);
                csub4(yy, make_float2(-w.x, -w.y), s4);
                y[e] = yy;
                float4 r4 = s4;
                csub4(r4, w, tv[e]);
                rr[e] = r4;
                facc_n2(acc, lo2(r4));
                facc_n2(acc, hi2(r4));
                facc_cdot(acc + 1, r0[e], r4);
            },
            W, sc + S_TS, s, 8.0 * n * 7));
        MGC_TRY(read_scalars(W, S_TS, 3, h, s));
        ++k;
        const double r2 = h[0];
        if (bad(r2)) return fail(MGC_ERR_BREAKDOWN, "QWS BiCGStab: non-finite residual");
        if (r2 <= tin * tin) break;
        const zd rho1(h[1], h[2]);
        if (rho == zd(0, 0) || omega == zd(0, 0)) break;
        const zd beta = (rho1 / rho) * (alpha / omega);
        const float2 bt = make_float2((float)beta.real(), (float)beta.imag());
        MGC_TRY(map32(
            n,
            [=] __device__(long long e) {
                float4 q = pv[e];
                csub4(q, w, v[e]);  // p - omega v
                float4 o = rr[e];
                csub4(o, make_float2(-bt.x, -bt.y), q);  // r + beta (p - omega v)
                pv[e] = o;
            },
            s, 8.0 * n * 3));
        rho = rho1;
    }
    *k_out = k;
    return MGC_OK;
}

static int qws(mgc_clover_s *op, const mgc_solve_params *p, mgc_solve_info *info, cudaStream_t s)
{
    SolverWork *W = op->work;
    const Geom &g = op->gauge->lat->g;
    const long long n = (long long)g.V * 12;
    double2 *x = W->x, *r = W->r, *b = W->b, *t = W->t;
    double *sc = W->scal;
    double bb, rr;
    MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, b[e]); }, W, sc + S_BB, s, 1));
    MGC_TRY(read_scalar(W, S_BB, &bb, s));
    info->iters = 0;
    info->restarts = 0;
    info->true_res = 0;
    if (bb == 0.0) {
        MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        return MGC_OK;
    }
    if (p->x_is_guess) {
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(residual(op, r, b, t, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
    } else {
        MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(double2), s));
        MGC_CUDA(cudaMemcpyAsync(r, b, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        rr = bb;
    }
    const double tol2 = p->tol * p->tol * bb;
    int iters = 0;
    for (;;) {
        info->true_res = std::sqrt(rr / bb);
        if (bad(rr)) return fail(MGC_ERR_BREAKDOWN, "QWS Richardson: non-finite residual");
        if (rr <= tol2) return MGC_OK;
        if (iters >= p->max_iter) return MGC_NOT_CONVERGED;
        // r_A = C^-1 r in FP64, its norm, and the unit-norm FP32 source
        MGC_TRY(launch_clover_apply(op, 64, true, r, t, 1, s));
        double ra2;
        MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, t[e]); }, W, sc + S_NW, s, 1));
        MGC_TRY(read_scalar(W, S_NW, &ra2, s));
        if (bad(ra2) || ra2 == 0.0) return fail(MGC_ERR_BREAKDOWN, "QWS Richardson: zero or non-finite C^-1 r");
        const double ra = std::sqrt(ra2);
        MGC_TRY(launch_scale_to32(g, t, W->r32, 1.0 / ra, s));
        double tin = p->inner_tol;
        const double need = 0.5 * p->tol * std::sqrt(bb / rr);
        if (need > tin) tin = need;
        int k = 0;
        MGC_TRY(inner_bicgstab32(op, p, tin, p->max_iter - iters, &k, s));
        iters += k;
        // x += ||r_A|| M y
        float2 *e32 = W->z32[3];
        MGC_TRY(precondition32_A(op, p, W->z32[2], e32, s));
        MGC_TRY(launch_axpy_from32(g, x, e32, ra, 0.0, s));
        MGC_TRY(apply_D64(op, x, t, s));
        MGC_TRY(residual(op, r, b, t, S_RR, s));
        MGC_TRY(read_scalar(W, S_RR, &rr, s));
        info->iters = iters;
        info->restarts++;
        MGC_TRY(check_device_status(op, s));
    }
}

// ------------------------------------------------------------------ entry points
static int check_params(const mgc_clover_s *op, const mgc_solve_params *p)
{
    if (p->method < 0 || p->method > 3)
        return fail(MGC_ERR_INVALID_ARG, "method must be 0 (FGCR), 1 (BiCGStab), 2 (two-level) or 3 (QWS)");
    if (p->method == 3 && (p->precond != 1 || p->smoother_prec == 64 || !has_prec(op->gauge, 32)))
        return fail(MGC_ERR_INVALID_ARG, "the QWS solve needs an FP32 copy, precond 1 and a 32- or 16-bit smoother");
    if (p->precond != 0 && p->precond != 1) return fail(MGC_ERR_INVALID_ARG, "precond must be 0 or 1");
    if (p->sap_solver != 0 && p->sap_solver != 2) return fail(MGC_ERR_INVALID_ARG, "sap_solver must be 0 or 2");
    if (p->precond == 1 && !has_prec(op->gauge, p->smoother_prec))
        return fail(MGC_ERR_INVALID_ARG, "no copy of the operator at smoother_prec");
    if (p->method == 2 && (!has_prec(op->gauge, 32) || (p->precond == 1 && p->smoother_prec == 64)))
        return fail(MGC_ERR_INVALID_ARG, "the two-level solve needs an FP32 copy and a 32- or 16-bit smoother");
    if (p->restart < 1 || p->restart > MAXM) return fail(MGC_ERR_INVALID_ARG, "restart must be in 1..32");
    if (!(p->tol > 0) || p->max_iter < 1 || p->n_cy < 0 || p->n_mr < 0 || !(p->inner_tol > 0))
        return fail(MGC_ERR_INVALID_ARG, "tol, inner_tol, max_iter, n_cy or n_mr out of range");
    return MGC_OK;
}

// The FP64 Krylov methods hand their vectors to an FP32 or FP16 smoother as
// they are.  For a source whose rms per real component lies beyond 2^+-30 they
// solve D (u x) = u b instead, u the power of two that brings that rms near 1
// (exact scaling: b and the guess are scaled in place, x back at the end), so
// that the smoother's sums of squares stay in FP32's range.  The two-level
// and QWS solves scale the residual of each outer step instead.
static int run_method(mgc_clover_s *op, const mgc_solve_params *p, mgc_solve_info *info, cudaStream_t s)
{
    if (p->method == 3) return qws(op, p, info, s);
    if (p->method == 2) return two_level(op, p, info, s);
    SolverWork *W = op->work;
    const long long n = (long long)op->gauge->lat->g.V * 12;
    double2 *x = W->x, *b = W->b;
    double u = 1.0;
    if (p->precond && p->smoother_prec != 64) {
        MGC_TRY(reduce<1>(n, [=] __device__(long long e, double *acc) { acc_n2(acc, b[e]); }, W, W->scal + S_BB, s, 1));
        double bb = 0.0;
        MGC_TRY(read_scalar(W, S_BB, &bb, s));
        const int e = unit_exp(bb, n);
        if (e > 30 || e < -30) {
            u = std::ldexp(1.0, e);
            const bool guess = p->x_is_guess != 0;
            MGC_TRY(map(
                n,
                [=] __device__(long long e) {
                    b[e] = make_double2(u * b[e].x, u * b[e].y);
                    if (guess) x[e] = make_double2(u * x[e].x, u * x[e].y);
                },
                s, guess ? 4 : 2));
        }
    }
    const int st = p->method == 0 ? fgcr(op, p, info, s) : fbicgstab(op, p, info, s);
    if (u != 1.0) {
        const double iu = 1.0 / u;
        MGC_TRY(map(
            n,
            [=] __device__(long long e) {
                x[e] = make_double2(iu * x[e].x, iu * x[e].y);
                b[e] = make_double2(iu * b[e].x, iu * b[e].y);
            },
            s, 4));
    }
    return st;
}

// ------------------------------------------------------------------ solve without allocation
// Scratch of mgc_solve_noalloc: a file-scope device array holding the
// flexible BiCGStab workspace (x, r, b, t, four w and four z FP64 vectors, two
// smoother buffers, reduction partials, scalars and the reduction ticket) for
// lattices of up to MGC_NOALLOC_MAX_SITES sites, about 10.5 MB.  Every GPU
// that loads the library holds it until the process exits.
constexpr size_t NA_VEC = (size_t)MGC_NOALLOC_MAX_SITES * 192;  // one FP64 packed spinor
constexpr size_t NA_LOW = (size_t)MGC_NOALLOC_MAX_SITES * 96;   // one FP32 or FP16 packed spinor
constexpr size_t NA_PART = (size_t)RGRID_MAX * PART_NV * sizeof(double);
constexpr size_t NA_SCAL = 1024;  // >= S_TOTAL doubles
constexpr size_t NA_CTR = 256;
constexpr size_t NA_BYTES = 12 * NA_VEC + 2 * NA_LOW + NA_PART + NA_SCAL + NA_CTR;
static_assert(NA_SCAL >= S_TOTAL * sizeof(double), "scalar area too small");
static __device__ __align__(256) unsigned char g_noalloc_scratch[NA_BYTES];

// device address of the scratch array, looked up once per device (in host
// code the array's name is only a stand-in, never a device address).  Atomic,
// so that two host threads making their first call at once both store the same
// address instead of racing on a plain pointer.
static std::atomic<void *> g_noalloc_base[64];
static double g_noalloc_hscal[2 * MAXM];  // pageable host copy of a few scalars

int solve_noalloc(mgc_clover_s *op, const double *b, double *x, const mgc_solve_params *p, mgc_solve_info *info,
                  cudaStream_t s)
{
    const Geom &g = op->gauge->lat->g;
    if (g.V > MGC_NOALLOC_MAX_SITES)
        return fail(MGC_ERR_UNSUPPORTED_SHAPE, "mgc_solve_noalloc: the lattice has more sites than "
                                               "MGC_NOALLOC_MAX_SITES (4096)");
    if (p->method != 1 || !p->on_device)
        return fail(MGC_ERR_INVALID_ARG,
                    "mgc_solve_noalloc: method must be 1 (flexible BiCGStab) and b, x device pointers");
    MGC_TRY(check_params(op, p));
    int dev = 0;
    MGC_CUDA(cudaGetDevice(&dev));
    if (dev < 0 || dev >= 64) return fail(MGC_ERR_INVALID_ARG, "mgc_solve_noalloc: device ordinal above 63");
    void *ptr = g_noalloc_base[dev].load(std::memory_order_acquire);
    if (!ptr) {
        MGC_CUDA(cudaGetSymbolAddress(&ptr, g_noalloc_scratch));
        g_noalloc_base[dev].store(ptr, std::memory_order_release);
    }
    unsigned char *base = static_cast<unsigned char *>(ptr);
    SolverWork W;  // a view of the scratch array: no allocation
    W.m = 4;
    W.lowprec = (p->precond && p->smoother_prec != 64) ? p->smoother_prec : 0;
    double2 **vec[12] = {&W.x, &W.r, &W.b, &W.t, &W.w[0], &W.w[1], &W.w[2], &W.w[3],
                         &W.z[0], &W.z[1], &W.z[2], &W.z[3]};
    for (int k = 0; k < 12; ++k) *vec[k] = reinterpret_cast<double2 *>(base + k * NA_VEC);
    unsigned char *q = base + 12 * NA_VEC;
    W.rl = q;
    W.zl = q + NA_LOW;
    q += 2 * NA_LOW;
    W.partial = reinterpret_cast<double *>(q);
    q += NA_PART;
    W.scal = reinterpret_cast<double *>(q);
    q += NA_SCAL;
    W.counter = reinterpret_cast<unsigned *>(q);
    W.hscal = g_noalloc_hscal;
    // the reduction ticket and the scalars must start at zero
    MGC_CUDA(cudaMemsetAsync(W.counter, 0, sizeof(unsigned), s));
    MGC_CUDA(cudaMemsetAsync(W.scal, 0, NA_SCAL, s));
    MGC_TRY(launch_pack(g, 64, 1, b, W.b, s));
    if (p->x_is_guess) MGC_TRY(launch_pack(g, 64, 1, x, W.x, s));
    mgc_solve_info one{MGC_OK, 0, 0, 0.0};
    SolverWork *saved = op->work;
    op->work = &W;
    const int st = fbicgstab(op, p, &one, s);
    op->work = saved;
    one.status = st;
    *info = one;
    if (st != MGC_OK && st != MGC_NOT_CONVERGED) return st;
    MGC_TRY(launch_unpack(g, 64, 1, W.x, x, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    return st;
}

int solve_packed(mgc_clover_s *op, const double2 *b, double2 *x, const mgc_solve_params *p, mgc_solve_info *info,
                 cudaStream_t s)
{
    MGC_TRY(check_params(op, p));
    MGC_TRY(ensure_work(op, p->method, p->restart, p->precond ? p->smoother_prec : 64));
    SolverWork *W = op->work;
    const size_t vb = spinor_bytes(op->gauge->lat->g, 64, 1);
    MGC_CUDA(cudaMemcpyAsync(W->b, b, vb, cudaMemcpyDeviceToDevice, s));
    if (p->x_is_guess) MGC_CUDA(cudaMemcpyAsync(W->x, x, vb, cudaMemcpyDeviceToDevice, s));
    const int st = run_method(op, p, info, s);
    info->status = st;
    MGC_CUDA(cudaMemcpyAsync(x, W->x, vb, cudaMemcpyDeviceToDevice, s));
    return st;
}

int solve(mgc_clover_s *op, const double *b, double *x, int nrhs, const mgc_solve_params *p, mgc_solve_info *info,
          cudaStream_t s)
{
    MGC_TRY(check_params(op, p));
    MGC_TRY(ensure_work(op, p->method, p->restart, p->precond ? p->smoother_prec : 64));
    SolverWork *W = op->work;
    const Geom &g = op->gauge->lat->g;
    const size_t vb = spinor_bytes(g, 64, 1);
    int worst = MGC_OK;
    mgc_solve_info agg{MGC_OK, 0, 0, 0.0};
    const bool next_b = !p->on_device && nrhs > 1 && page_locked(b);
    if (next_b && !W->stage2) MGC_CUDA(cudaMalloc(&W->stage2, vb));
    bool b_waiting = false;  // stage2 receives this right-hand side's b (ev_b)
    for (int k = 0; k < nrhs; ++k) {
        const double *bk = b + (size_t)k * g.V * 24;
        double *xk = x + (size_t)k * g.V * 24;
        if (p->on_device) {
            MGC_TRY(launch_pack(g, 64, 1, bk, W->b, s));
            if (p->x_is_guess) MGC_TRY(launch_pack(g, 64, 1, xk, W->x, s));
        } else {
            const double2 *src = W->stage;
            if (b_waiting) {
                MGC_CUDA(cudaStreamWaitEvent(s, W->ev_b, 0));
                src = W->stage2;
                b_waiting = false;
            } else {
                MGC_CUDA(cudaMemcpyAsync(W->stage, bk, vb, cudaMemcpyHostToDevice, s));
            }
            MGC_TRY(launch_pack(g, 64, 1, (const double *)src, W->b, s));
            if (next_b && k + 1 < nrhs) {
                // the next b crosses the host link while this one is solved,
                // into stage2 once the pack above has read it
                MGC_CUDA(cudaEventRecord(W->ev_x, s));
                MGC_CUDA(cudaStreamWaitEvent(W->copy_stream, W->ev_x, 0));
                MGC_CUDA(cudaMemcpyAsync(W->stage2, bk + (size_t)g.V * 24, vb, cudaMemcpyHostToDevice,
                                         W->copy_stream));
                MGC_CUDA(cudaEventRecord(W->ev_b, W->copy_stream));
                b_waiting = true;
            }
            if (p->x_is_guess) {
                MGC_CUDA(cudaMemcpyAsync(W->stage, xk, vb, cudaMemcpyHostToDevice, s));
                MGC_TRY(launch_pack(g, 64, 1, (const double *)W->stage, W->x, s));
            }
        }
        mgc_solve_info one{MGC_OK, 0, 0, 0.0};
        W->host_x = (!p->on_device && page_locked(xk)) ? xk : nullptr;
        const int st = run_method(op, p, &one, s);
        W->host_x = nullptr;
        if (st != MGC_OK && st != MGC_NOT_CONVERGED) {
            // no copy from the caller's b or into its x may still run after the return
            cudaStreamSynchronize(W->copy_stream);
            W->copy_live = false;
            one.status = st;
            *info = one;
            return st;
        }
        if (p->on_device) {
            MGC_TRY(launch_unpack(g, 64, 1, W->x, xk, s));
        } else if (W->copy_live && st == MGC_OK) {
            MGC_TRY(join_copy(W, s));  // the converged x is on its way to the host
        } else {
            MGC_TRY(join_copy(W, s));
            MGC_TRY(launch_unpack(g, 64, 1, W->x, (double *)W->stage, s));
            MGC_CUDA(cudaMemcpyAsync(xk, W->stage, vb, cudaMemcpyDeviceToHost, s));
        }
        if (st != MGC_OK) worst = st;
        agg.iters = one.iters > agg.iters ? one.iters : agg.iters;
        agg.restarts += one.restarts;
        agg.true_res = one.true_res > agg.true_res ? one.true_res : agg.true_res;
    }
    MGC_CUDA(cudaStreamSynchronize(s));
    agg.status = worst;
    *info = agg;
    return worst;
}

}  // namespace mgc
