// Batches of lattices: one launch per step over every right-hand side of
// every lattice of the batch.
//
//   - mgc_batch_apply_D: the multi-RHS Dslash (Eq. (1)) over all lattices, in
//     the launch shape the autotuner picked.
//   - mgc_batch_sap_smooth: the multiplicative SAP smoother (Sec. 2) over all
//     lattices, 2 n_cy launches captured once into a CUDA graph and replayed.
//   - mgc_batch_solve: the two-level solve (FP64 defect correction, the
//     Richardson iteration of Sec. 2, around an FP32 FGCR inner solve
//     preconditioned by SAP, Sec. 3) for all systems in lock step.  Every
//     system keeps its own Krylov coefficients in device memory; one inner
//     iteration of all systems is one CUDA graph (smoother, D, the
//     orthogonalisation and the updates) followed by a single 4-byte read of
//     "is any system still iterating".
//
// Vectors of the batched solve are flat: lattice k's nrhs[k] packed fields sit
// back to back at offset off[k] (complex elements), so system s (operator
// major) is one contiguous segment.  Reductions are segmented: each thread
// block covers up to BCHUNK elements of a single system and a second kernel
// sums each system's block partials in a fixed order, so results are
// deterministic.
#include <algorithm>
#include <cmath>
#include <cstddef>
#include <cstring>
#include <vector>

#include "mgc_host.h"

namespace mgc {
namespace {

constexpr int BRT = 256;       // threads of the segmented kernels
// elements per segmented block: 64 per thread, so the block's FP64 reduction
// of up to 16 accumulators is amortised over enough data (with 16 per thread
// the Gram-Schmidt pass ran at a quarter of HBM bandwidth)
constexpr int BCHUNK = 16384;
constexpr int BMAXM = 16;      // longest inner cycle of the batched solve
constexpr int BCH32 = 16;      // FP32 accumulation chunk
constexpr int SU = 4;          // elements per thread per step of the segmented kernels

// per-system scalars of the batched solve
struct SysScal {
    double bb, rr64, rr, nw, true_res, tin2;
    double rho[2];
    double d[2 * (BMAXM + 1)];  // <L_i, w_j>: L_i = w'_i (i < j), then r
    double n2[BMAXM];
    double R[BMAXM][BMAXM][2];
    double alpha[BMAXM][2];
    double gamma[BMAXM][2];
    float coef[BMAXM][2];
    float g32[BMAXM][2];
    float a32[2];
    int active, k, iters, restarts, status, pad;
};
static_assert(sizeof(SysScal) % sizeof(double) == 0, "SysScal must be a whole number of doubles");
constexpr int SSTRIDE = sizeof(SysScal) / sizeof(double);

// address of a double field of system 0 (the others follow at SSTRIDE)
inline double *sfield(SysScal *S, size_t offset) { return (double *)((char *)S + offset); }

struct SegTab {
    const int *blk_sys;
    const int *sys_blk0;  // nsys + 1 entries
    const long long *sys_off;
    const int *sys_len;
};

template <int NV>
__device__ __forceinline__ void bblock_reduce(double *v, double (*sh)[BRT / 32])
{
#pragma unroll
    for (int k = 0; k < NV; ++k)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) v[k] += __shfl_xor_sync(0xffffffffu, v[k], o);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) sh[k][warp] = v[k];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) {
            double s = 0;
            for (int w = 0; w < BRT / 32; ++w) s += sh[k][w];
            v[k] = s;
        }
}

__device__ __forceinline__ void seg_range(const SegTab &t, int &s, long long &start, long long &end)
{
    const int b = blockIdx.x;
    s = t.blk_sys[b];
    const long long base = t.sys_off[s];
    start = base + (long long)(b - t.sys_blk0[s]) * BCHUNK;
    end = base + t.sys_len[s];
    if (end > start + BCHUNK) end = start + BCHUNK;
}

// partial[b][k] = sum over the elements of block b of what f accumulates;
// FP32 functors accumulate BCH32 elements in FP32, then in FP64
template <int NV, bool F32, class F>
__global__ void __launch_bounds__(BRT) k_seg_reduce(SegTab t, F f, double *partial)
{
    static_assert(NV <= 16, "the batch partial-sum area holds sixteen accumulators per block");
    __shared__ double sh[NV][BRT / 32];
    int s;
    long long start, end;
    seg_range(t, s, start, end);
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0;
    if constexpr (F32) {
        float facc[NV];
#pragma unroll
        for (int k = 0; k < NV; ++k) facc[k] = 0.f;
        // SU independent elements per step (BRT apart, so a warp's loads stay
        // contiguous) keep enough loads in flight to cover HBM latency
        int c = 0;
        long long e = start + threadIdx.x;
        for (; e + (SU - 1) * BRT < end; e += SU * BRT) {
#pragma unroll
            for (int u = 0; u < SU; ++u) f(e + u * BRT, s, facc);
            c += SU;
            if (c >= BCH32) {
                c = 0;
#pragma unroll
                for (int k = 0; k < NV; ++k) {
                    acc[k] += (double)facc[k];
                    facc[k] = 0.f;
                }
            }
        }
        for (; e < end; e += BRT) f(e, s, facc);
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += (double)facc[k];
    } else {
        long long e = start + threadIdx.x;
        for (; e + (SU - 1) * BRT < end; e += SU * BRT)
#pragma unroll
            for (int u = 0; u < SU; ++u) f(e + u * BRT, s, acc);
        for (; e < end; e += BRT) f(e, s, acc);
    }
    bblock_reduce<NV>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) partial[(size_t)blockIdx.x * NV + k] = acc[k];
}

// out[s * stride + k] = sum of system s's block partials, in block order
template <int NV>
__global__ void __launch_bounds__(BRT) k_seg_finish(SegTab t, const double *partial, double *out, int stride)
{
    __shared__ double sh[NV][BRT / 32];
    const int s = blockIdx.x;
    double acc[NV];
#pragma unroll
    for (int k = 0; k < NV; ++k) acc[k] = 0;
    for (int b = t.sys_blk0[s] + threadIdx.x; b < t.sys_blk0[s + 1]; b += BRT)
#pragma unroll
        for (int k = 0; k < NV; ++k) acc[k] += partial[(size_t)b * NV + k];
    bblock_reduce<NV>(acc, sh);
    if (threadIdx.x == 0)
#pragma unroll
        for (int k = 0; k < NV; ++k) out[(size_t)s * stride + k] = acc[k];
}

template <class F>
__global__ void __launch_bounds__(BRT) k_seg_map(SegTab t, F f)
{
    int s;
    long long start, end;
    seg_range(t, s, start, end);
    long long e = start + threadIdx.x;
    for (; e + (SU - 1) * BRT < end; e += SU * BRT)
#pragma unroll
        for (int u = 0; u < SU; ++u) f(e + u * BRT, s);
    for (; e < end; e += BRT) f(e, s);
}

__device__ __forceinline__ void fdot(float *acc, float2 a, float2 b)
{
    acc[0] = fmaf(a.x, b.x, fmaf(a.y, b.y, acc[0]));
    acc[1] = fmaf(a.x, b.y, fmaf(-a.y, b.x, acc[1]));
}
__device__ __forceinline__ void fn2(float *acc, float2 a) { acc[0] = fmaf(a.x, a.x, fmaf(a.y, a.y, acc[0])); }
__device__ __forceinline__ void dn2(double *acc, double2 a) { acc[0] = fma(a.x, a.x, fma(a.y, a.y, acc[0])); }

struct Ptr8 {
    const float2 *p[8];
};
struct PtrM {
    const float2 *p[BMAXM];
};

// ---- per-system scalar steps (one thread per system)
__global__ void k_sc_start(SysScal *S, int n, int from_bb)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    if (from_bb) S[s].rr64 = S[s].bb;
    S[s].iters = 0;
    S[s].restarts = 0;
    S[s].status = MGC_OK;
    S[s].true_res = 0;
}

__global__ void k_sc_outer(SysScal *S, int n, double tol, double inner_tol, int max_iter, double *rnorm,
                           double *inv_rnorm, int *act, int *flags)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SysScal &q = S[s];
    const double bb = q.bb, rr = q.rr64;
    q.true_res = bb > 0 ? sqrt(rr / bb) : 0.0;
    int a = 0;
    if (q.status == MGC_OK && bb > 0) {
        if (!isfinite(rr)) q.status = MGC_ERR_BREAKDOWN;
        else if (rr <= tol * tol * bb) a = 0;
        else if (q.iters >= max_iter) q.status = MGC_NOT_CONVERGED;
        else a = 1;
    }
    act[s] = a;
    q.active = a;
    q.k = 0;
    if (a) {
        const double rn = sqrt(rr);
        rnorm[s] = rn;
        inv_rnorm[s] = 1.0 / rn;
        double tin = 0.5 * tol * sqrt(bb / rr);
        if (tin < inner_tol) tin = inner_tol;
        q.tin2 = tin * tin;
        atomicOr(flags, 1);
    } else {
        rnorm[s] = 0;
        inv_rnorm[s] = 0;
    }
}

// c_i = <w'_i, w_j> / ||w'_i||^2 for i < j; rho = <w_j, r>
__global__ void k_sc_orth(SysScal *S, int n, int j)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SysScal &q = S[s];
    q.rho[0] = q.d[2 * j];
    q.rho[1] = -q.d[2 * j + 1];
    for (int i = 0; i < j; ++i) {
        const double n2 = q.n2[i];
        const double cr = n2 > 0 ? q.d[2 * i] / n2 : 0.0, ci = n2 > 0 ? q.d[2 * i + 1] / n2 : 0.0;
        q.R[i][j][0] = cr;
        q.R[i][j][1] = ci;
        q.coef[i][0] = (float)cr;
        q.coef[i][1] = (float)ci;
    }
}

__global__ void k_sc_alpha(SysScal *S, int n, int j)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SysScal &q = S[s];
    const double nw = q.nw;
    q.n2[j] = nw;
    double ar = 0, ai = 0;
    if (q.active) {
        if (nw > 0 && isfinite(nw)) {
            ar = q.rho[0] / nw;
            ai = q.rho[1] / nw;
        } else {
            q.status = MGC_ERR_BREAKDOWN;
            q.active = 0;
        }
    }
    q.alpha[j][0] = ar;
    q.alpha[j][1] = ai;
    q.a32[0] = (float)ar;
    q.a32[1] = (float)ai;
}

__global__ void k_sc_conv(SysScal *S, int n, int j, int *flags)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SysScal &q = S[s];
    if (!q.active) return;
    q.k = j + 1;
    const double rr = q.rr;
    if (!isfinite(rr)) {
        q.status = MGC_ERR_BREAKDOWN;
        q.active = 0;
    } else if (rr <= q.tin2) {
        q.active = 0;
    }
    if (q.active) atomicOr(flags, 1);
}

// R gamma = alpha (R unit upper triangular, R_ij = c_ij) over the k directions
__global__ void k_sc_gamma(SysScal *S, int n, const int *act)
{
    const int s = blockIdx.x * blockDim.x + threadIdx.x;
    if (s >= n) return;
    SysScal &q = S[s];
    const int k = q.k;
    for (int i = BMAXM - 1; i >= 0; --i) {
        double gr = 0, gi = 0;
        if (i < k) {
            gr = q.alpha[i][0];
            gi = q.alpha[i][1];
            for (int jj = i + 1; jj < k; ++jj) {
                const double rr = q.R[i][jj][0], ri = q.R[i][jj][1];
                const double xr = q.gamma[jj][0], xi = q.gamma[jj][1];
                gr -= rr * xr - ri * xi;
                gi -= rr * xi + ri * xr;
            }
        }
        q.gamma[i][0] = gr;
        q.gamma[i][1] = gi;
        q.g32[i][0] = (float)gr;
        q.g32[i][1] = (float)gi;
    }
    q.iters += k;
    if (act[s]) q.restarts++;
}

inline int sc_grid(int n) { return (n + 127) / 128; }

}  // namespace

// ------------------------------------------------------------------ workspace
struct BatchWork {
    int m = 0, lowprec = 0;
    double2 *x = nullptr, *r = nullptr, *b = nullptr, *t = nullptr, *stage = nullptr;
    float2 *r32 = nullptr, *w32[BMAXM] = {}, *z32[BMAXM] = {};
    unsigned char *rl = nullptr, *zl = nullptr;  // FP16 smoother fields, per lattice at loff16
    size_t loff16[MGC_BATCH_MAX] = {};
    SysScal *S = nullptr;
    double *rnorm = nullptr, *inv_rnorm = nullptr;
    int *act = nullptr;
    int *flags = nullptr;   // device: [0] any system iterating
    int *hflags = nullptr;  // pinned host copy
    double *partial = nullptr;
    int *blk_sys = nullptr, *sys_blk0 = nullptr, *sys_len = nullptr;
    long long *sys_off = nullptr;
    int nblk = 0;
    // graphs of the inner iterations, valid for key
    int key[6] = {-1, -1, -1, -1, -1, -1};
    cudaGraphExec_t iter_graph[BMAXM] = {};
    long long iter_launches[BMAXM] = {};
    double iter_bytes[BMAXM] = {};
};

}  // namespace mgc

using namespace mgc;

struct BatchTune {
    int done = 0, rb = 1, threads = 256, rf_d = 1, rf_sap = 1;
};

struct SapGraph {
    int prec, n_cy, n_mr, xz, rf;
    std::vector<const void *> b;
    std::vector<void *> x;
    cudaGraphExec_t exec;
    long long launches;
    double bytes;
};

struct mgc_batch_s {
    BatchSpec spec;
    int nsys = 0;
    size_t off[MGC_BATCH_MAX] = {};  // flat offsets (complex elements)
    size_t ntot = 0;
    cudaStream_t cap = nullptr;      // private stream for capture and tuning
    BatchTune tune[3];               // prec 64, 32, 16
    std::vector<SapGraph> sap_graphs;
    BatchWork *work = nullptr;
};

namespace {

int prec_slot(int prec) { return prec == 64 ? 0 : (prec == 32 ? 1 : 2); }

void release_graphs(mgc_batch_s *B)
{
    for (auto &g : B->sap_graphs) cudaGraphExecDestroy(g.exec);
    B->sap_graphs.clear();
    if (B->work)
        for (int j = 0; j < BMAXM; ++j)
            if (B->work->iter_graph[j]) {
                cudaGraphExecDestroy(B->work->iter_graph[j]);
                B->work->iter_graph[j] = nullptr;
            }
}

void free_batch_work(BatchWork *W)
{
    if (!W) return;
    for (int j = 0; j < BMAXM; ++j)
        if (W->iter_graph[j]) cudaGraphExecDestroy(W->iter_graph[j]);
    void *dev[] = {W->x, W->r, W->b, W->t, W->stage, W->r32, W->rl, W->zl, W->S, W->rnorm, W->inv_rnorm, W->act,
                   W->flags, W->partial, W->blk_sys, W->sys_blk0, W->sys_len, W->sys_off};
    for (void *p : dev)
        if (p) cudaFree(p);
    for (int j = 0; j < BMAXM; ++j) {
        if (W->w32[j]) cudaFree(W->w32[j]);
        if (W->z32[j]) cudaFree(W->z32[j]);
    }
    if (W->hflags) cudaFreeHost(W->hflags);
    delete W;
}

// capture what body enqueues on the private stream into an executable graph;
// the library counters keep what one replay adds, not the capture itself
template <class F>
int capture(cudaStream_t cap, F body, cudaGraphExec_t *exec, long long *nl, double *nb)
{
    long long l0, l1;
    double b0, b1;
    mgc_counters(&l0, &b0, 0);
    MGC_CUDA(cudaStreamBeginCapture(cap, cudaStreamCaptureModeRelaxed));
    const int st = body(cap);
    cudaGraph_t graph = nullptr;
    const cudaError_t e = cudaStreamEndCapture(cap, &graph);
    mgc_counters(&l1, &b1, 0);
    count(-(l1 - l0), -(b1 - b0));
    *nl = l1 - l0;
    *nb = b1 - b0;
    if (st != MGC_OK) {
        if (graph) cudaGraphDestroy(graph);
        return st;
    }
    if (e != cudaSuccess) return cuda_fail(e, "cudaStreamEndCapture", __FILE__, __LINE__);
    const cudaError_t ei = cudaGraphInstantiate(exec, graph, 0);
    cudaGraphDestroy(graph);
    if (ei != cudaSuccess) return cuda_fail(ei, "cudaGraphInstantiate", __FILE__, __LINE__);
    return MGC_OK;
}

int replay(cudaGraphExec_t exec, long long nl, double nb, cudaStream_t s)
{
    MGC_CUDA(cudaGraphLaunch(exec, s));
    count(nl, nb);
    return MGC_OK;
}

bool capturing(cudaStream_t s)
{
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(s, &cs) != cudaSuccess) {
        cudaGetLastError();
        return true;
    }
    return cs != cudaStreamCaptureStatusNone;
}

BatchSpec spec_with(const mgc_batch_s *B, int rf)
{
    BatchSpec sp = B->spec;
    sp.rhs_fast = rf;
    return sp;
}

// time the launch shapes of D (and the smoother block order) on scratch fields
int run_tune(mgc_batch_s *B, int prec)
{
    BatchTune &T = B->tune[prec_slot(prec)];
    const int n = B->spec.n;
    int maxr = 1;
    for (int k = 0; k < n; ++k) maxr = std::max(maxr, B->spec.nrhs[k]);
    size_t offs[MGC_BATCH_MAX], tot = 0;
    for (int k = 0; k < n; ++k) {
        offs[k] = tot;
        tot += (spinor_bytes(B->spec.ops[k]->gauge->lat->g, prec, B->spec.nrhs[k]) + 255) / 256 * 256;
    }
    unsigned char *bin = nullptr, *bout = nullptr;
    MGC_CUDA(cudaMalloc(&bin, tot));
    if (cudaMalloc(&bout, tot) != cudaSuccess) {
        cudaFree(bin);
        return fail(MGC_ERR_CUDA, "autotuner: out of device memory");
    }
    const void *in[MGC_BATCH_MAX];
    void *out[MGC_BATCH_MAX];
    for (int k = 0; k < n; ++k) {
        in[k] = bin + offs[k];
        out[k] = bout + offs[k];
    }
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    long long l0, l1;
    double b0, b1;
    mgc_counters(&l0, &b0, 0);
    int st = MGC_OK;
    cudaStream_t s = B->cap;
    // byte 0x3c gives small finite non-zero values in every storage format
    if (cudaMemsetAsync(bin, 0x3c, tot, s) != cudaSuccess || cudaEventCreate(&e0) != cudaSuccess ||
        cudaEventCreate(&e1) != cudaSuccess)
        st = fail(MGC_ERR_CUDA, "autotuner: setup failed");
    auto timed = [&](auto launch, int reps, float *ms) -> int {
        MGC_TRY(launch());
        MGC_CUDA(cudaEventRecord(e0, s));
        for (int r = 0; r < reps; ++r) MGC_TRY(launch());
        MGC_CUDA(cudaEventRecord(e1, s));
        MGC_CUDA(cudaEventSynchronize(e1));
        MGC_CUDA(cudaEventElapsedTime(ms, e0, e1));
        return MGC_OK;
    };
    float best = 1e30f;
    const int rbs[3] = {1, 2, 4};
    for (int a = 0; a < 3 && st == MGC_OK; ++a) {
        const int rb = rbs[a];
        if (rb > 1 && (rb + 1) / 2 >= maxr) continue;  // 2 needs >= 2 rhs, 4 needs >= 3
        for (int threads = 128; threads <= 256 && st == MGC_OK; threads *= 2)
            for (int rf = 0; rf <= 1 && st == MGC_OK; ++rf) {
                if (rf == 1 && maxr <= rb) continue;  // one group per site block: the order is the same
                const BatchSpec sp = spec_with(B, rf);
                float ms = 0;
                st = timed([&]() { return launch_dirac_batch(sp, prec, false, in, out, rb, threads, s); }, 3, &ms);
                if (st == MGC_OK && ms < best) {
                    best = ms;
                    T.rb = rb;
                    T.threads = threads;
                    T.rf_d = rf;
                }
            }
    }
    if (st == MGC_OK && prec != 64) {
        float bs = 1e30f;
        for (int rf = 0; rf <= 1 && st == MGC_OK; ++rf) {
            const BatchSpec sp = spec_with(B, rf);
            float ms = 0;
            st = timed(
                [&]() -> int {
                    MGC_CUDA(cudaMemsetAsync(bout, 0, tot, s));
                    return launch_sap_batch(sp, prec, in, out, 1, 4, 1, s);
                },
                2, &ms);
            if (st == MGC_OK && ms < bs) {
                bs = ms;
                T.rf_sap = rf;
            }
        }
    }
    cudaStreamSynchronize(s);
    mgc_counters(&l1, &b1, 0);
    count(-(l1 - l0), -(b1 - b0));
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    cudaFree(bin);
    cudaFree(bout);
    if (st == MGC_OK) T.done = 1;
    return st;
}

// tuned shape, tuning now unless the caller's stream is being captured
int get_tune(mgc_batch_s *B, int prec, cudaStream_t s, BatchTune *out)
{
    BatchTune &T = B->tune[prec_slot(prec)];
    if (!T.done && !capturing(s)) {
        MGC_CUDA(cudaStreamSynchronize(s));
        MGC_TRY(run_tune(B, prec));
    }
    *out = T;
    return MGC_OK;
}

int check_fields(const mgc_batch_s *B, const void *const *a, const void *const *b)
{
    if (!B || !a || !b) return fail(MGC_ERR_INVALID_ARG, "null batch or field array");
    for (int k = 0; k < B->spec.n; ++k) {
        if (!a[k] || !b[k]) return fail(MGC_ERR_INVALID_ARG, "null field pointer");
        if (a[k] == b[k]) return fail(MGC_ERR_INVALID_ARG, "input and output fields must not overlap");
    }
    return MGC_OK;
}

int batch_has_prec(const mgc_batch_s *B, int prec)
{
    if (prec != 64 && prec != 32 && prec != 16) return fail(MGC_ERR_INVALID_ARG, "prec must be 64, 32 or 16");
    if (!has_prec(B->spec.ops[0]->gauge, prec))
        return fail(MGC_ERR_INVALID_ARG, "the operators keep no copy at this precision");
    return MGC_OK;
}

// ------------------------------------------------------------------ batched solve
template <int NV, bool F32, class F>
int seg_reduce(const mgc_batch_s *B, F f, double *out, int stride, cudaStream_t s, double bytes)
{
    const BatchWork *W = B->work;
    const SegTab t{W->blk_sys, W->sys_blk0, W->sys_off, W->sys_len};
    k_seg_reduce<NV, F32><<<W->nblk, BRT, 0, s>>>(t, f, W->partial);
    k_seg_finish<NV><<<B->nsys, BRT, 0, s>>>(t, W->partial, out, stride);
    MGC_CUDA(cudaGetLastError());
    count(2, bytes);
    return MGC_OK;
}

template <int NV, class F>
int seg_reduce32(const mgc_batch_s *B, F f, double *out, int stride, cudaStream_t s, double bytes)
{
    return seg_reduce<NV, true>(B, f, out, stride, s, bytes);
}

template <int NV, class F>
int seg_reduce64(const mgc_batch_s *B, F f, double *out, int stride, cudaStream_t s, double bytes)
{
    return seg_reduce<NV, false>(B, f, out, stride, s, bytes);
}

template <class F>
int seg_map(const mgc_batch_s *B, F f, cudaStream_t s, double bytes)
{
    const BatchWork *W = B->work;
    const SegTab t{W->blk_sys, W->sys_blk0, W->sys_off, W->sys_len};
    k_seg_map<<<W->nblk, BRT, 0, s>>>(t, f);
    MGC_CUDA(cudaGetLastError());
    count(1, bytes);
    return MGC_OK;
}

template <class T>
int dalloc(T **p, size_t bytes)
{
    MGC_CUDA(cudaMalloc((void **)p, bytes));
    return MGC_OK;
}

int ensure_batch_work(mgc_batch_s *B, int m, int lowprec)
{
    BatchWork *W = B->work;
    if (W && W->m >= m && (lowprec != 16 || W->lowprec == 16)) return MGC_OK;
    if (W) {
        free_batch_work(W);
        B->work = nullptr;
    }
    W = new BatchWork();
    B->work = W;
    W->m = m;
    W->lowprec = lowprec;
    const size_t n = B->ntot;
    MGC_TRY(dalloc(&W->x, n * sizeof(double2)));
    MGC_TRY(dalloc(&W->r, n * sizeof(double2)));
    MGC_TRY(dalloc(&W->b, n * sizeof(double2)));
    MGC_TRY(dalloc(&W->t, n * sizeof(double2)));
    MGC_TRY(dalloc(&W->stage, n * sizeof(double2)));
    MGC_TRY(dalloc(&W->r32, n * sizeof(float2)));
    for (int j = 0; j < m; ++j) {
        MGC_TRY(dalloc(&W->w32[j], n * sizeof(float2)));
        MGC_TRY(dalloc(&W->z32[j], n * sizeof(float2)));
    }
    if (lowprec == 16) {
        size_t tot = 0;
        for (int k = 0; k < B->spec.n; ++k) {
            W->loff16[k] = tot;
            tot += (spinor_bytes(B->spec.ops[k]->gauge->lat->g, 16, B->spec.nrhs[k]) + 255) / 256 * 256;
        }
        MGC_TRY(dalloc(&W->rl, tot));
        MGC_TRY(dalloc(&W->zl, tot));
    }
    const int ns = B->nsys;
    MGC_TRY(dalloc(&W->S, ns * sizeof(SysScal)));
    MGC_CUDA(cudaMemset(W->S, 0, ns * sizeof(SysScal)));
    MGC_TRY(dalloc(&W->rnorm, ns * sizeof(double)));
    MGC_TRY(dalloc(&W->inv_rnorm, ns * sizeof(double)));
    MGC_TRY(dalloc(&W->act, ns * sizeof(int)));
    MGC_TRY(dalloc(&W->flags, 4 * sizeof(int)));
    MGC_CUDA(cudaMallocHost((void **)&W->hflags, 4 * sizeof(int)));
    // segmentation: each system is one run of BCHUNK-element blocks
    std::vector<int> blk_sys, blk0(ns + 1), len(ns);
    std::vector<long long> soff(ns);
    int sys = 0;
    for (int k = 0; k < B->spec.n; ++k) {
        const int V = B->spec.ops[k]->gauge->lat->g.V;
        for (int q = 0; q < B->spec.nrhs[k]; ++q, ++sys) {
            soff[sys] = (long long)B->off[k] + (long long)q * V * 12;
            len[sys] = V * 12;
            blk0[sys] = (int)blk_sys.size();
            const int nb = (len[sys] + BCHUNK - 1) / BCHUNK;
            for (int b = 0; b < nb; ++b) blk_sys.push_back(sys);
        }
    }
    blk0[ns] = (int)blk_sys.size();
    W->nblk = (int)blk_sys.size();
    MGC_TRY(dalloc(&W->partial, (size_t)W->nblk * 16 * sizeof(double)));
    MGC_TRY(dalloc(&W->blk_sys, blk_sys.size() * sizeof(int)));
    MGC_TRY(dalloc(&W->sys_blk0, blk0.size() * sizeof(int)));
    MGC_TRY(dalloc(&W->sys_len, len.size() * sizeof(int)));
    MGC_TRY(dalloc(&W->sys_off, soff.size() * sizeof(long long)));
    MGC_CUDA(cudaMemcpy(W->blk_sys, blk_sys.data(), blk_sys.size() * sizeof(int), cudaMemcpyHostToDevice));
    MGC_CUDA(cudaMemcpy(W->sys_blk0, blk0.data(), blk0.size() * sizeof(int), cudaMemcpyHostToDevice));
    MGC_CUDA(cudaMemcpy(W->sys_len, len.data(), len.size() * sizeof(int), cudaMemcpyHostToDevice));
    MGC_CUDA(cudaMemcpy(W->sys_off, soff.data(), soff.size() * sizeof(long long), cudaMemcpyHostToDevice));
    return MGC_OK;
}

// per-lattice pointers into a flat batch vector
template <class T>
void lattice_ptrs(const mgc_batch_s *B, T *flat, T **out)
{
    for (int k = 0; k < B->spec.n; ++k) out[k] = flat + B->off[k];
}

// one inner FGCR iteration j of every system (what the graph of j holds)
int inner_step(mgc_batch_s *B, const mgc_solve_params *p, const BatchTune &T32, const BatchTune &Ts, int j,
               cudaStream_t s)
{
    BatchWork *W = B->work;
    const size_t n = B->ntot;
    const double dn = (double)n * 8.0;  // bytes of one FP32 flat vector
    SysScal *S = W->S;
    const int ns = B->nsys;
    float2 *r = W->r32, *zj = W->z32[j], *wj = W->w32[j];
    MGC_CUDA(cudaMemsetAsync(W->flags, 0, sizeof(int), s));
    MGC_CUDA(cudaMemsetAsync(zj, 0, n * sizeof(float2), s));
    // z_j = M_SAP r
    float2 *rk[MGC_BATCH_MAX], *zk[MGC_BATCH_MAX];
    lattice_ptrs(B, r, rk);
    lattice_ptrs(B, zj, zk);
    const BatchSpec ssap = spec_with(B, Ts.rf_sap);
    if (p->smoother_prec == 32) {
        MGC_TRY(launch_sap_batch(ssap, 32, (const void *const *)rk, (void *const *)zk, p->n_cy, p->n_mr, 1, s));
    } else {
        const void *rl[MGC_BATCH_MAX];
        void *zl[MGC_BATCH_MAX];
        size_t tot = 0;
        for (int k = 0; k < B->spec.n; ++k) {
            const Geom &g = B->spec.ops[k]->gauge->lat->g;
            rl[k] = W->rl + W->loff16[k];
            zl[k] = W->zl + W->loff16[k];
            tot = W->loff16[k] + spinor_bytes(g, 16, B->spec.nrhs[k]);
            MGC_TRY(launch_convert(g, B->spec.nrhs[k], 32, rk[k], 16, (void *)rl[k], s));
        }
        MGC_CUDA(cudaMemsetAsync(W->zl, 0, tot, s));
        MGC_TRY(launch_sap_batch(ssap, 16, rl, zl, p->n_cy, p->n_mr, 1, s));
        for (int k = 0; k < B->spec.n; ++k)
            MGC_TRY(launch_convert(B->spec.ops[k]->gauge->lat->g, B->spec.nrhs[k], 16, zl[k], 32, zk[k], s));
    }
    // w_j = D z_j
    float2 *wk[MGC_BATCH_MAX];
    lattice_ptrs(B, wj, wk);
    MGC_TRY(launch_dirac_batch(spec_with(B, T32.rf_d), 32, false, (const void *const *)zk, (void *const *)wk, T32.rb,
                               T32.threads, s));
    // d_i = <L_i, w_j>, L = (w'_0 .. w'_{j-1}, r), eight per pass
    for (int i0 = 0; i0 <= j; i0 += 8) {
        const int cnt = std::min(8, j + 1 - i0);
        Ptr8 L{};
        for (int q = 0; q < cnt; ++q) L.p[q] = (i0 + q < j) ? W->w32[i0 + q] : r;
        const float2 *wv = wj;
        MGC_TRY(seg_reduce32<16>(
            B,
            [=] __device__(long long e, int, float *acc) {
                const float2 v = wv[e];
#pragma unroll
                for (int q = 0; q < 8; ++q)
                    if (q < cnt) fdot(acc + 2 * q, L.p[q][e], v);
            },
            sfield(S, offsetof(SysScal, d)) + 2 * i0, SSTRIDE, s, dn * (cnt + 1)));
    }
    k_sc_orth<<<sc_grid(ns), 128, 0, s>>>(S, ns, j);
    // w'_j = w_j - sum_i c_i w'_i and its norm
    PtrM Lw{};
    for (int i = 0; i < j; ++i) Lw.p[i] = W->w32[i];
    MGC_TRY(seg_reduce32<1>(
        B,
        [=] __device__(long long e, int sys, float *acc) {
            float2 v = wj[e];
            const SysScal &q = S[sys];
            for (int i = 0; i < j; ++i) {
                const float cx = q.coef[i][0], cy = q.coef[i][1];
                const float2 u = Lw.p[i][e];
                v.x -= cx * u.x - cy * u.y;
                v.y -= cx * u.y + cy * u.x;
            }
            wj[e] = v;
            fn2(acc, v);
        },
        sfield(S, offsetof(SysScal, nw)), SSTRIDE, s, dn * (j + 2)));
    k_sc_alpha<<<sc_grid(ns), 128, 0, s>>>(S, ns, j);
    // r -= alpha_j w'_j and ||r||^2
    MGC_TRY(seg_reduce32<1>(
        B,
        [=] __device__(long long e, int sys, float *acc) {
            const float ax = S[sys].a32[0], ay = S[sys].a32[1];
            const float2 u = wj[e];
            float2 v = r[e];
            v.x -= ax * u.x - ay * u.y;
            v.y -= ax * u.y + ay * u.x;
            r[e] = v;
            fn2(acc, v);
        },
        sfield(S, offsetof(SysScal, rr)), SSTRIDE, s, dn * 3));
    k_sc_conv<<<sc_grid(ns), 128, 0, s>>>(S, ns, j, W->flags);
    MGC_CUDA(cudaGetLastError());
    count(3, 0);
    MGC_CUDA(cudaMemcpyAsync(W->hflags, W->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
    return MGC_OK;
}

int read_flag(const BatchWork *W, cudaStream_t s, int *v)
{
    MGC_CUDA(cudaStreamSynchronize(s));
    *v = W->hflags[0];
    return MGC_OK;
}

// r = b - D x (FP64) and ||r||^2 per system
int batch_residual(mgc_batch_s *B, const BatchTune &T64, cudaStream_t s)
{
    BatchWork *W = B->work;
    double2 *xk[MGC_BATCH_MAX], *tk[MGC_BATCH_MAX];
    lattice_ptrs(B, W->x, xk);
    lattice_ptrs(B, W->t, tk);
    MGC_TRY(launch_dirac_batch(spec_with(B, T64.rf_d), 64, false, (const void *const *)xk, (void *const *)tk, T64.rb,
                               T64.threads, s));
    double2 *r = W->r, *t = W->t;
    const double2 *b = W->b;
    return seg_reduce64<1>(
        B,
        [=] __device__(long long e, int, double *acc) {
            const double2 v = make_double2(b[e].x - t[e].x, b[e].y - t[e].y);
            r[e] = v;
            dn2(acc, v);
        },
        sfield(W->S, offsetof(SysScal, rr64)), SSTRIDE, s, (double)B->ntot * 16.0 * 3);
}

int batch_two_level(mgc_batch_s *B, const mgc_solve_params *p, cudaStream_t s)
{
    BatchWork *W = B->work;
    const int ns = B->nsys;
    const size_t n = B->ntot;
    BatchTune T64, T32, Ts;
    MGC_TRY(get_tune(B, 64, s, &T64));
    MGC_TRY(get_tune(B, 32, s, &T32));
    Ts = T32;
    if (p->smoother_prec == 16) {
        BatchTune T16;
        MGC_TRY(get_tune(B, 16, s, &T16));
        Ts.rf_sap = T16.rf_sap;
    }
    // inner-iteration graphs depend on these
    const int key[6] = {p->n_cy, p->n_mr, p->smoother_prec, T32.rb * 1000 + T32.threads, T32.rf_d, Ts.rf_sap};
    if (std::memcmp(key, W->key, sizeof(key)) != 0) {
        for (int j = 0; j < BMAXM; ++j)
            if (W->iter_graph[j]) {
                cudaGraphExecDestroy(W->iter_graph[j]);
                W->iter_graph[j] = nullptr;
            }
        std::memcpy(W->key, key, sizeof(key));
    }
    SysScal *S = W->S;
    const double2 *b = W->b;
    MGC_TRY(seg_reduce64<1>(
        B, [=] __device__(long long e, int, double *acc) { dn2(acc, b[e]); }, sfield(S, offsetof(SysScal, bb)), SSTRIDE, s,
        (double)n * 16.0));
    if (p->x_is_guess) {
        k_sc_start<<<sc_grid(ns), 128, 0, s>>>(S, ns, 0);
        // a system with b = 0 has the solution 0 whatever the guess
        double2 *x = W->x;
        MGC_TRY(seg_map(
            B,
            [=] __device__(long long e, int sys) {
                if (S[sys].bb == 0.0) x[e] = make_double2(0.0, 0.0);
            },
            s, (double)n * 16.0));
        MGC_TRY(batch_residual(B, T64, s));
    } else {
        MGC_CUDA(cudaMemsetAsync(W->x, 0, n * sizeof(double2), s));
        MGC_CUDA(cudaMemcpyAsync(W->r, W->b, n * sizeof(double2), cudaMemcpyDeviceToDevice, s));
        k_sc_start<<<sc_grid(ns), 128, 0, s>>>(S, ns, 1);
    }
    MGC_CUDA(cudaGetLastError());
    const int m = std::min(p->restart, BMAXM);
    for (;;) {
        MGC_CUDA(cudaMemsetAsync(W->flags, 0, sizeof(int), s));
        k_sc_outer<<<sc_grid(ns), 128, 0, s>>>(S, ns, p->tol, p->inner_tol, p->max_iter, W->rnorm, W->inv_rnorm,
                                               W->act, W->flags);
        MGC_CUDA(cudaGetLastError());
        count(1, 0);
        MGC_CUDA(cudaMemcpyAsync(W->hflags, W->flags, sizeof(int), cudaMemcpyDeviceToHost, s));
        int any = 0;
        MGC_TRY(read_flag(W, s, &any));
        if (!any) break;
        // r32 = r / ||r|| for the systems still iterating, 0 for the others
        MGC_TRY(launch_scale_to32_batch(B->spec, B->off, W->r, W->r32, W->inv_rnorm, W->act, s));
        int jmax = 0;
        for (int j = 0; j < m; ++j) {
            if (!W->iter_graph[j]) {
                MGC_TRY(capture(
                    B->cap, [&](cudaStream_t cs) { return inner_step(B, p, T32, Ts, j, cs); }, &W->iter_graph[j],
                    &W->iter_launches[j], &W->iter_bytes[j]));
            }
            MGC_TRY(replay(W->iter_graph[j], W->iter_launches[j], W->iter_bytes[j], s));
            jmax = j + 1;
            MGC_TRY(read_flag(W, s, &any));
            if (!any) break;
        }
        k_sc_gamma<<<sc_grid(ns), 128, 0, s>>>(S, ns, W->act);
        count(1, 0);
        // e = sum_j gamma_j z_j (FP32, into w32[0]), then x += ||r|| e in FP64
        PtrM Lz{};
        for (int j = 0; j < jmax; ++j) Lz.p[j] = W->z32[j];
        float2 *esum = W->w32[0];
        MGC_TRY(seg_map(
            B,
            [=] __device__(long long e, int sys) {
                const SysScal &q = S[sys];
                float sx = 0.f, sy = 0.f;
                for (int j = 0; j < jmax; ++j) {
                    const float cx = q.g32[j][0], cy = q.g32[j][1];
                    const float2 z = Lz.p[j][e];
                    sx += cx * z.x - cy * z.y;
                    sy += cx * z.y + cy * z.x;
                }
                esum[e] = make_float2(sx, sy);
            },
            s, (double)n * 8.0 * (jmax + 1)));
        MGC_TRY(launch_axpy_from32_batch(B->spec, B->off, W->x, esum, W->rnorm, W->act, s));
        MGC_TRY(batch_residual(B, T64, s));
        for (int k = 0; k < B->spec.n; ++k) MGC_TRY(check_device_status(B->spec.ops[k], s));
    }
    return MGC_OK;
}

}  // namespace

// ------------------------------------------------------------------ C ABI
extern "C" {

int mgc_batch_create(const mgc_clover_t *ops, const int *nrhs, int n, mgc_batch_t *out)
{
    if (!ops || !nrhs || !out || n < 1 || n > MGC_BATCH_MAX) return fail(MGC_ERR_INVALID_ARG, "bad batch arguments");
    *out = nullptr;
    const mgc_gauge_s *g0 = ops[0] ? ops[0]->gauge : nullptr;
    if (!g0) return fail(MGC_ERR_INVALID_ARG, "null operator");
    for (int k = 0; k < n; ++k) {
        if (!ops[k] || nrhs[k] < 1) return fail(MGC_ERR_INVALID_ARG, "null operator or nrhs < 1");
        const mgc_gauge_s *g = ops[k]->gauge;
        if (g->prec != g0->prec || g->compress != g0->compress)
            return fail(MGC_ERR_INVALID_ARG, "operators of a batch must share storage precision and compression");
        for (int mu = 0; mu < 4; ++mu)
            if (g->lat->g.lb[mu] != g0->lat->g.lb[mu])
                return fail(MGC_ERR_UNSUPPORTED_SHAPE, "operators of a batch must share the SAP domain shape");
    }
    mgc_batch_s *B = new mgc_batch_s();
    B->spec.n = n;
    B->spec.rhs_fast = 1;
    size_t tot = 0;
    for (int k = 0; k < n; ++k) {
        B->spec.ops[k] = ops[k];
        B->spec.nrhs[k] = nrhs[k];
        B->off[k] = tot;
        tot += (size_t)ops[k]->gauge->lat->g.V * 12 * nrhs[k];
        B->nsys += nrhs[k];
    }
    B->ntot = tot;
    const cudaError_t e = cudaStreamCreateWithFlags(&B->cap, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
        delete B;
        return cuda_fail(e, "cudaStreamCreateWithFlags", __FILE__, __LINE__);
    }
    *out = B;
    return ok();
}

int mgc_batch_destroy(mgc_batch_t B)
{
    if (!B) return MGC_OK;
    cudaDeviceSynchronize();
    release_graphs(B);
    free_batch_work(B->work);
    if (B->cap) cudaStreamDestroy(B->cap);
    delete B;
    return ok();
}

int mgc_batch_systems(mgc_batch_t B) { return B ? B->nsys : 0; }

int mgc_batch_apply_D(mgc_batch_t B, const void *const *in, void *const *out, int prec, int dagger, void *stream)
{
    MGC_TRY(check_fields(B, in, (const void *const *)out));
    MGC_TRY(batch_has_prec(B, prec));
    const cudaStream_t s = (cudaStream_t)stream;
    BatchTune T;
    MGC_TRY(get_tune(B, prec, s, &T));
    return launch_dirac_batch(spec_with(B, T.rf_d), prec, dagger != 0, in, out, T.rb, T.threads, s);
}

int mgc_batch_sap_smooth(mgc_batch_t B, const void *const *rhs, void *const *x, int n_cy, int n_mr, int prec,
                         int x_is_zero, void *stream)
{
    MGC_TRY(check_fields(B, rhs, (const void *const *)x));
    if (prec != 32 && prec != 16) return fail(MGC_ERR_INVALID_ARG, "batched smoother precision must be 32 or 16");
    MGC_TRY(batch_has_prec(B, prec));
    if (n_cy < 0 || n_mr < 0) return fail(MGC_ERR_INVALID_ARG, "n_cy and n_mr must be >= 0");
    const cudaStream_t s = (cudaStream_t)stream;
    BatchTune T;
    MGC_TRY(get_tune(B, prec, s, &T));
    const BatchSpec sp = spec_with(B, T.rf_sap);
    const int xz = x_is_zero ? 1 : 0;
    if (n_cy == 0) return ok();
    if (capturing(s)) return launch_sap_batch(sp, prec, rhs, x, n_cy, n_mr, xz, s);
    const int n = B->spec.n;
    for (auto &gr : B->sap_graphs) {
        if (gr.prec != prec || gr.n_cy != n_cy || gr.n_mr != n_mr || gr.xz != xz || gr.rf != T.rf_sap) continue;
        bool same = true;
        for (int k = 0; k < n; ++k) same = same && gr.b[k] == rhs[k] && gr.x[k] == x[k];
        if (same) return replay(gr.exec, gr.launches, gr.bytes, s);
    }
    SapGraph gr{prec, n_cy, n_mr, xz, T.rf_sap, std::vector<const void *>(rhs, rhs + n),
                std::vector<void *>(x, x + n), nullptr, 0, 0.0};
    MGC_TRY(capture(
        B->cap, [&](cudaStream_t cs) { return launch_sap_batch(sp, prec, rhs, x, n_cy, n_mr, xz, cs); }, &gr.exec,
        &gr.launches, &gr.bytes));
    if (B->sap_graphs.size() >= 4) {
        cudaGraphExecDestroy(B->sap_graphs.front().exec);
        B->sap_graphs.erase(B->sap_graphs.begin());
    }
    B->sap_graphs.push_back(gr);
    return replay(gr.exec, gr.launches, gr.bytes, s);
}

int mgc_batch_tune(mgc_batch_t B, int prec, int force, int *rhs_per_thread, int *threads, int *rhs_fast_d,
                   int *rhs_fast_sap, void *stream)
{
    if (!B) return fail(MGC_ERR_INVALID_ARG, "null batch");
    MGC_TRY(batch_has_prec(B, prec));
    const cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return fail(MGC_ERR_INVALID_ARG, "cannot tune while the stream is being captured");
    if (force) B->tune[prec_slot(prec)].done = 0;
    BatchTune T;
    MGC_TRY(get_tune(B, prec, s, &T));
    if (rhs_per_thread) *rhs_per_thread = T.rb;
    if (threads) *threads = T.threads;
    if (rhs_fast_d) *rhs_fast_d = T.rf_d;
    if (rhs_fast_sap) *rhs_fast_sap = T.rf_sap;
    return ok();
}

int mgc_batch_set_shape(mgc_batch_t B, int prec, int rhs_per_thread, int threads, int rhs_fast_d, int rhs_fast_sap)
{
    if (!B) return fail(MGC_ERR_INVALID_ARG, "null batch");
    MGC_TRY(batch_has_prec(B, prec));
    if ((rhs_per_thread != 1 && rhs_per_thread != 2 && rhs_per_thread != 4) || (threads != 128 && threads != 256) ||
        (rhs_fast_d != 0 && rhs_fast_d != 1) || (rhs_fast_sap != 0 && rhs_fast_sap != 1))
        return fail(MGC_ERR_INVALID_ARG, "bad launch shape");
    BatchTune &T = B->tune[prec_slot(prec)];
    T.rb = rhs_per_thread;
    T.threads = threads;
    T.rf_d = rhs_fast_d;
    T.rf_sap = rhs_fast_sap;
    T.done = 1;
    return ok();
}

int mgc_batch_solve(mgc_batch_t B, const double *const *rhs, double *const *x, const mgc_solve_params *p,
                    mgc_solve_info *info, void *stream)
{
    if (!B || !rhs || !x || !p || !info) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    for (int k = 0; k < B->spec.n; ++k)
        if (!rhs[k] || !x[k]) return fail(MGC_ERR_INVALID_ARG, "null field pointer");
    if (p->method != 2 || p->precond != 1)
        return fail(MGC_ERR_INVALID_ARG, "the batched solve is the two-level method with SAP (method 2, precond 1)");
    if (p->smoother_prec != 32 && p->smoother_prec != 16)
        return fail(MGC_ERR_INVALID_ARG, "smoother_prec must be 32 or 16");
    if (p->sap_solver != 0) return fail(MGC_ERR_INVALID_ARG, "the batched solve uses the MR domain solver (sap_solver 0)");
    if (!has_prec(B->spec.ops[0]->gauge, p->smoother_prec) || !has_prec(B->spec.ops[0]->gauge, 32))
        return fail(MGC_ERR_INVALID_ARG, "the operators keep no copy at the smoother precision");
    if (p->restart < 1 || p->n_cy < 1 || p->n_mr < 1 || !(p->tol > 0) || p->max_iter < 1 || !(p->inner_tol > 0))
        return fail(MGC_ERR_INVALID_ARG, "bad solver parameters");
    const cudaStream_t s = (cudaStream_t)stream;
    if (capturing(s)) return fail(MGC_ERR_INVALID_ARG, "mgc_batch_solve synchronises: the stream must not be captured");
    MGC_TRY(ensure_batch_work(B, std::min(p->restart, BMAXM), p->smoother_prec));
    BatchWork *W = B->work;
    // pack the right-hand sides (and guesses) into the flat FP64 vectors
    for (int k = 0; k < B->spec.n; ++k) {
        const Geom &g = B->spec.ops[k]->gauge->lat->g;
        const int nr = B->spec.nrhs[k];
        const size_t bytes = (size_t)g.V * 12 * nr * sizeof(double2);
        const double *srcs[2] = {rhs[k], x[k]};
        double2 *dsts[2] = {W->b + B->off[k], W->x + B->off[k]};
        for (int w = 0; w < (p->x_is_guess ? 2 : 1); ++w) {
            const double *src = srcs[w];
            if (!p->on_device) {
                MGC_CUDA(cudaMemcpyAsync(W->stage + B->off[k], src, bytes, cudaMemcpyHostToDevice, s));
                src = (const double *)(W->stage + B->off[k]);
            }
            MGC_TRY(launch_pack(g, 64, nr, src, dsts[w], s));
        }
    }
    const int st = batch_two_level(B, p, s);
    if (st != MGC_OK) return st;
    for (int k = 0; k < B->spec.n; ++k) {
        const Geom &g = B->spec.ops[k]->gauge->lat->g;
        const int nr = B->spec.nrhs[k];
        if (p->on_device) {
            MGC_TRY(launch_unpack(g, 64, nr, W->x + B->off[k], x[k], s));
        } else {
            MGC_TRY(launch_unpack(g, 64, nr, W->x + B->off[k], (double *)(W->stage + B->off[k]), s));
            MGC_CUDA(cudaMemcpyAsync(x[k], W->stage + B->off[k], (size_t)g.V * 12 * nr * sizeof(double2),
                                     cudaMemcpyDeviceToHost, s));
        }
    }
    std::vector<SysScal> hs(B->nsys);
    MGC_CUDA(cudaMemcpyAsync(hs.data(), W->S, B->nsys * sizeof(SysScal), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    int worst = MGC_OK;
    for (int i = 0; i < B->nsys; ++i) {
        info[i].status = hs[i].status;
        info[i].iters = hs[i].iters;
        info[i].restarts = hs[i].restarts;
        info[i].true_res = hs[i].true_res;
        if (hs[i].status == MGC_ERR_BREAKDOWN) worst = MGC_ERR_BREAKDOWN;
        else if (hs[i].status != MGC_OK && worst == MGC_OK) worst = hs[i].status;
    }
    if (worst == MGC_ERR_BREAKDOWN) return fail(worst, "batched solve: breakdown in at least one system");
    return worst == MGC_OK ? ok() : worst;
}

}  // extern "C"
