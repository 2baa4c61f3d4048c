// Multiplicative Schwarz alternating procedure (Sec. 2: QWS's M_SAP, used as
// the post-smoother of Sec. 3), one kernel launch per colour of domains.
//
// One thread block per domain B of the current colour, one thread per site:
//   1. r_B = (b - D x)|_B with the full operator (the other colour's x on the
//      faces comes from global memory); skipped (r_B = b_B) when x == 0;
//   2. n_mr minimal-residual steps on the Dirichlet domain operator D_B from
//      e = 0:  p = D_B r, alpha = <p, r>/<p, p>, e += alpha r, r -= alpha p,
//      with r held in shared memory and the three inner products reduced by
//      warp shuffles and one shared-memory pass;
//   3. x_B += e.
// Domains of one colour never touch each other, so the launches of a sweep
// are red then black and every block of a launch is independent.
#include "hop.cuh"
#include "mgc_host.h"

namespace mgc {

// sum of three values over the thread block, identical on every thread
template <typename T>
__device__ __forceinline__ void block_sum3(T &a, T &b, T &c, T *red)
{
    const int nt = blockDim.x;
    const unsigned mask = nt >= 32 ? 0xffffffffu : ((1u << nt) - 1u);
    const int width = nt >= 32 ? 32 : nt;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        if (o < width) {
            a += __shfl_xor_sync(mask, a, o);
            b += __shfl_xor_sync(mask, b, o);
            c += __shfl_xor_sync(mask, c, o);
        }
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp] = a;
        red[32 + warp] = b;
        red[64 + warp] = c;
    }
    __syncthreads();
    const int nw = (nt + 31) >> 5;
    a = 0;
    b = 0;
    c = 0;
    for (int w = 0; w < nw; ++w) {
        a += red[w];
        b += red[32 + w];
        c += red[64 + w];
    }
}

// p = D_B r at local site l, r from shared memory rs[12][Vb]
template <int MU, class GA, typename T>
__device__ __forceinline__ void block_hop_dir(const GA &U, int blkbase, int i, int nf, int nb, const Cx<T> *rs,
                                              int vb, Cx<T> acc[12])
{
    Cx<T> s[12], h[6], w[6], u[9];
    if (nf >= 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = rs[k * vb + nf];
        project<MU, -1>(s, h);
        U.load(i, MU, u);
        su3_mul(u, h, w);
        reconstruct_add<MU, -1>(acc, w);
    }
    if (nb >= 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = rs[k * vb + nb];
        project<MU, +1>(s, h);
        U.load(blkbase + nb, MU, u);
        su3_dag_mul(u, h, w);
        reconstruct_add<MU, +1>(acc, w);
    }
}

template <class SP, class GA, class CL>
__global__ void __launch_bounds__(256) k_sap_colour(Geom g, SP b, SP x, GA U, CL C, typename SP::Real kappa,
                                                    int colour, int nmr, int x_zero)
{
    using T = typename SP::Real;
    extern __shared__ __align__(16) unsigned char smem[];
    const int vb = 1 << g.lvb;
    Cx<T> *rs = reinterpret_cast<Cx<T> *>(smem);
    T *red = reinterpret_cast<T *>(rs + 12 * vb);

    const int r = blockIdx.y;
    const SP bb = shift_rhs(b, r, g.V);
    const SP xx = shift_rhs(x, r, g.V);

    // the domain of this thread block: the blockIdx.x-th domain of `colour`
    int j = blockIdx.x;
    const int half0 = g.NB[0] >> 1;
    int bc[4];
    const int m = j % half0;
    j /= half0;
    bc[1] = j % g.NB[1];
    j /= g.NB[1];
    bc[2] = j % g.NB[2];
    bc[3] = j / g.NB[2];
    bc[0] = 2 * m + ((colour + bc[1] + bc[2] + bc[3]) & 1);
    const int blkbase = block_index(g, bc) << g.lvb;
    const int l = threadIdx.x;
    const int i = blkbase | l;
    int lc[4], c[4];
    local_coords(g, l, lc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) c[mu] = (bc[mu] << g.lb[mu]) + lc[mu];

    // 1. block residual
    Cx<T> rv[12];
    bb.load(i, rv);
    if (!x_zero) {
        Cx<T> dx[12];
        dirac_site<false>(g, c, i, xx, U, C, kappa, dx);
#pragma unroll
        for (int k = 0; k < 12; ++k) rv[k] = rv[k] - dx[k];
    }
    // in-domain neighbours (local index, or -1 when the hop leaves the domain)
    int nf[4], nb[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int t[4] = {lc[0], lc[1], lc[2], lc[3]};
        t[mu] = lc[mu] + 1;
        nf[mu] = (t[mu] < (1 << g.lb[mu])) ? local_index(g, t) : -1;
        t[mu] = lc[mu] - 1;
        nb[mu] = (t[mu] >= 0) ? local_index(g, t) : -1;
    }
#pragma unroll
    for (int k = 0; k < 12; ++k) rs[k * vb + l] = rv[k];
    Cx<T> e[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = Cx<T>{0, 0};
    __syncthreads();

    // 2. minimal residual on D_B
    for (int it = 0; it < nmr; ++it) {
        Cx<T> acc[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = Cx<T>{0, 0};
        block_hop_dir<0>(U, blkbase, i, nf[0], nb[0], rs, vb, acc);
        block_hop_dir<1>(U, blkbase, i, nf[1], nb[1], rs, vb, acc);
        block_hop_dir<2>(U, blkbase, i, nf[2], nb[2], rs, vb, acc);
        block_hop_dir<3>(U, blkbase, i, nf[3], nb[3], rs, vb, acc);
        T cl[72];
        C.load(i, cl);
        Cx<T> p[12];
        clover_mul(cl, rv, p);
        T pr = 0, pi = 0, pp = 0;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k] = Cx<T>{fma(-kappa, acc[k].r, p[k].r), fma(-kappa, acc[k].i, p[k].i)};
            pr = fma(p[k].r, rv[k].r, fma(p[k].i, rv[k].i, pr));
            pi = fma(p[k].r, rv[k].i, fma(-p[k].i, rv[k].r, pi));
            pp = fma(p[k].r, p[k].r, fma(p[k].i, p[k].i, pp));
        }
        block_sum3(pr, pi, pp, red);
        const Cx<T> alpha = (pp > 0) ? Cx<T>{pr / pp, pi / pp} : Cx<T>{0, 0};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            e[k] = cfma(alpha, rv[k], e[k]);
            rv[k] = rv[k] - alpha * p[k];
            rs[k * vb + l] = rv[k];
        }
        __syncthreads();
    }

    // 3. x_B += e
    if (!x_zero) {
        Cx<T> xo[12];
        xx.load(i, xo);
#pragma unroll
        for (int k = 0; k < 12; ++k) e[k] = e[k] + xo[k];
    }
    xx.store(i, e);
}

// Algorithmic bytes of one colour's launch over its V/2 sites: b, the
// domains' links and clover, x written, and, unless x == 0, x of the domains
// and of the other colour read.
static double sap_launch_bytes(const Geom &g, int prec, int compress, int nrhs, bool xz)
{
    const double sp = spinor_site_bytes(prec);
    return 0.5 * g.V * (nrhs * (sp + sp + (xz ? 0.0 : 2.0 * sp)) + links_site_bytes(prec, compress) +
                        clover_site_bytes(prec));
}

template <class SP, class GA, class CL>
static int sap_run(const Geom &g, SP b, SP x, GA U, CL C, double kappa, int nrhs, int n_cy, int n_mr, int x_is_zero,
                   cudaStream_t s, int prec, int compress)
{
    using T = typename SP::Real;
    const int vb = 1 << g.lvb;
    const size_t smem = (size_t)vb * 12 * sizeof(Cx<T>) + 96 * sizeof(T);
    auto kern = k_sap_colour<SP, GA, CL>;
    if (smem > 48 * 1024) MGC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(g.nblocks / 2, nrhs);
    for (int cy = 0; cy < n_cy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int xz = (cy == 0 && colour == 0) ? x_is_zero : 0;
            kern<<<grid, vb, smem, s>>>(g, b, x, U, C, (T)kappa, colour, n_mr, xz);
            count(1, sap_launch_bytes(g, prec, compress, nrhs, xz != 0));
        }
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

int launch_sap(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_mr, int x_is_zero,
               cudaStream_t s)
{
    const mgc_gauge_s *ga = op->gauge;
    const Geom &g = ga->lat->g;
    if ((1 << g.lvb) > 256) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "SAP domains are limited to 256 sites");
    if (prec == 64) {
        return sap_run(g, Spinor64{(double2 *)b, g.lvb}, Spinor64{(double2 *)x, g.lvb}, Gauge64{ga->U64, g.lvb},
                       Clover64{op->C64, g.lvb}, op->kappa, nrhs, n_cy, n_mr, x_is_zero, s, prec, ga->compress);
    }
    if (prec != ga->prec) return fail(MGC_ERR_INVALID_ARG, "smoother precision differs from the gauge storage precision");
    if (prec == 32) {
        Spinor32 B{(float4 *)b, g.lvb}, X{(float4 *)x, g.lvb};
        Clover32 C{(float4 *)op->Clo, g.lvb};
        if (ga->compress == 12) return sap_run(g, B, X, Gauge32x12{(float4 *)ga->Ulo, g.lvb}, C, op->kappa, nrhs, n_cy, n_mr, x_is_zero, s, prec, ga->compress);
        return sap_run(g, B, X, Gauge32x18{(float2 *)ga->Ulo, g.lvb}, C, op->kappa, nrhs, n_cy, n_mr, x_is_zero, s, prec, ga->compress);
    }
    const size_t nV = (size_t)nrhs * g.V;
    Spinor16 B{(uint4 *)b, (float *)((uint4 *)b + nV * 3), g.lvb};
    Spinor16 X{(uint4 *)x, (float *)((uint4 *)x + nV * 3), g.lvb};
    Clover16 C{(uint4 *)op->Clo, op->Clo_sc, g.lvb};
    if (ga->compress == 12) return sap_run(g, B, X, Gauge16x12{(uint2 *)ga->Ulo, g.lvb}, C, op->kappa, nrhs, n_cy, n_mr, x_is_zero, s, prec, ga->compress);
    return sap_run(g, B, X, Gauge16x18{(uint32_t *)ga->Ulo, g.lvb}, C, op->kappa, nrhs, n_cy, n_mr, x_is_zero, s, prec, ga->compress);
}

}  // namespace mgc
