// Batches of lattices: the dispatch of the batched multi-RHS D (kernels in
// dirac_batch.cuh, instantiated per storage precision) and the per-system
// FP64 <-> FP32 site kernels of the batched two-level solve.
#include "dirac_batch.cuh"

namespace mgc {

int launch_dirac_batch(const BatchSpec &spec, int prec, bool dag, const void *const *in, void *const *out, int rb,
                       int threads, cudaStream_t s)
{
    if (rb != 1 && rb != 2 && rb != 4) return fail(MGC_ERR_INVALID_ARG, "right-hand sides per thread must be 1, 2 or 4");
    if (threads != 128 && threads != 256) return fail(MGC_ERR_INVALID_ARG, "threads per block must be 128 or 256");
    const mgc_gauge_s *ga0 = spec.ops[0]->gauge;
    double bytes = 0;
    for (int k = 0; k < spec.n; ++k) {
        const Geom &g = spec.ops[k]->gauge->lat->g;
        bytes += (double)g.V * (2.0 * spec.nrhs[k] * spinor_site_bytes(prec) +
                                links_site_bytes(prec, prec == 64 ? 18 : ga0->compress) + clover_site_bytes(prec));
    }
    const int st = prec == 64   ? dirac_batch_64(spec, dag, in, out, rb, threads, s)
                   : prec == 32 ? dirac_batch_32(spec, dag, in, out, rb, threads, s)
                                : dirac_batch_16(spec, dag, in, out, rb, threads, s);
    if (st == MGC_OK) count(1, bytes);
    return st;
}

// per-system FP64 <-> FP32 site kernels of the batched solve: thread block b
// covers 256 sites of one right-hand side of one lattice
struct SiteBatch {
    int n;
    int end[MGC_BATCH_MAX];
    int nsb[MGC_BATCH_MAX];
    int sys0[MGC_BATCH_MAX];
    Geom g[MGC_BATCH_MAX];
    size_t off[MGC_BATCH_MAX];
};

static int site_batch(const BatchSpec &spec, const size_t *off, SiteBatch &B, double *bytes, double per_site)
{
    B.n = spec.n;
    int acc = 0, sys = 0;
    *bytes = 0;
    for (int k = 0; k < spec.n; ++k) {
        const Geom &g = spec.ops[k]->gauge->lat->g;
        B.g[k] = g;
        B.nsb[k] = grid_for(g.V, 256);
        B.sys0[k] = sys;
        B.off[k] = off[k];
        sys += spec.nrhs[k];
        acc += B.nsb[k] * spec.nrhs[k];
        B.end[k] = acc;
        *bytes += (double)g.V * spec.nrhs[k] * per_site;
    }
    return acc;
}

__device__ __forceinline__ bool site_item(const SiteBatch &B, int &k, int &q, int &i)
{
    k = 0;
    while (k < B.n - 1 && (int)blockIdx.x >= B.end[k]) ++k;
    const int local = blockIdx.x - (k ? B.end[k - 1] : 0);
    q = local / B.nsb[k];
    i = (local % B.nsb[k]) * 256 + threadIdx.x;
    return i < B.g[k].V;
}

__global__ void __launch_bounds__(256) k_scale_to32_batch(SiteBatch B, const double2 *in, float2 *out,
                                                          const double *scal, const int *flag)
{
    int k, q, i;
    if (!site_item(B, k, q, i)) return;
    const Geom &g = B.g[k];
    const int sys = B.sys0[k] + q;
    const double f = flag[sys] ? scal[sys] : 0.0;
    Spinor64 a = shift_rhs(Spinor64{(double2 *)in + B.off[k], g.lvb}, q, g.V);
    Spinor32 o = shift_rhs(Spinor32{(float4 *)(out + B.off[k]), g.lvb}, q, g.V);
    Cx<double> v[12];
    Cx<float> w[12];
    a.load(i, v);
#pragma unroll
    for (int c = 0; c < 12; ++c) w[c] = Cx<float>{(float)(f * v[c].r), (float)(f * v[c].i)};
    o.store(i, w);
}

__global__ void __launch_bounds__(256) k_axpy_from32_batch(SiteBatch B, double2 *x, const float2 *e,
                                                           const double *scal, const int *flag)
{
    int k, q, i;
    if (!site_item(B, k, q, i)) return;
    const Geom &g = B.g[k];
    const int sys = B.sys0[k] + q;
    if (!flag[sys]) return;
    const double f = scal[sys];
    Spinor64 a = shift_rhs(Spinor64{x + B.off[k], g.lvb}, q, g.V);
    Spinor32 d = shift_rhs(Spinor32{(float4 *)(e + B.off[k]), g.lvb}, q, g.V);
    Cx<double> v[12];
    Cx<float> w[12];
    a.load(i, v);
    d.load(i, w);
#pragma unroll
    for (int c = 0; c < 12; ++c) v[c] = Cx<double>{fma(f, (double)w[c].r, v[c].r), fma(f, (double)w[c].i, v[c].i)};
    a.store(i, v);
}

int launch_scale_to32_batch(const BatchSpec &spec, const size_t *off, const double2 *in, float2 *out,
                            const double *scal, const int *flag, cudaStream_t s)
{
    SiteBatch B;
    double bytes;
    const int grid = site_batch(spec, off, B, &bytes, 192.0 + 96.0);
    k_scale_to32_batch<<<grid, 256, 0, s>>>(B, in, out, scal, flag);
    MGC_CUDA(cudaGetLastError());
    count(1, bytes);
    return MGC_OK;
}

int launch_axpy_from32_batch(const BatchSpec &spec, const size_t *off, double2 *x, const float2 *e,
                             const double *scal, const int *flag, cudaStream_t s)
{
    SiteBatch B;
    double bytes;
    const int grid = site_batch(spec, off, B, &bytes, 2 * 192.0 + 96.0);
    k_axpy_from32_batch<<<grid, 256, 0, s>>>(B, x, e, scal, flag);
    MGC_CUDA(cudaGetLastError());
    count(1, bytes);
    return MGC_OK;
}

}  // namespace mgc
