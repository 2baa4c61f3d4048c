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
//
// In mode SAP_JAC the same kernels run QWS's smoother for the clover-
// preconditioned operator A = C^-1 D = 1 - kappa C^-1 H (Sec. 2): the staged
// clover term is C^-1, the domain residual is r_B = (b - x + kappa C^-1 H x)|_B,
// and the domain solve is a fixed number n_j of Jacobi iterations
// e <- r_B + kappa C^-1 H_B e from e = 0 (the first gives e = r_B), with e
// (instead of r) in shared memory and no block reductions.
//
// In mode SAP_EO (FP64 and staged kernels) the domain solve is the even-odd
// preconditioned MR of DD-alphaAMG: the even sites (the first half of a domain
// in the packed order) run MR on the Schur complement
// C_ee - kappa^2 H_eo C_oo^-1 H_oe with source r_e + kappa H_eo C_oo^-1 r_o,
// the odd sites apply C_oo^-1 (read from global memory) in between and finally
// form e_o = C_oo^-1 (r_o + kappa H_oe e_e).  Odd entries of the shared vector
// hold the odd-site intermediate, even entries the even-site residual.
#include "hop.cuh"
#include "hop16.cuh"
#include "mgc_host.h"
#include "tma.cuh"

namespace mgc {

// domain solvers of the smoother kernels: MR on D_B; Jacobi on A_B (QWS);
// even-odd preconditioned MR on D_B (MR on the even Schur complement)
enum { SAP_MR = 0, SAP_JAC = 1, SAP_EO = 2 };

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

// block_sum3 for blocks of NT threads, NT a multiple of 128, with float
// partials in a 16-byte aligned red: the warps' partials read back as float4
template <int NT>
__device__ __forceinline__ void block_sum3_v4(float &a, float &b, float &c, float *red)
{
    static_assert(NT % 128 == 0, "four warps per float4 of partials");
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        a += __shfl_xor_sync(0xffffffffu, a, o);
        b += __shfl_xor_sync(0xffffffffu, b, o);
        c += __shfl_xor_sync(0xffffffffu, c, o);
    }
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) {
        red[warp] = a;
        red[32 + warp] = b;
        red[64 + warp] = c;
    }
    __syncthreads();
    const float4 *r4 = reinterpret_cast<const float4 *>(red);
    float4 sa = r4[0], sb = r4[8], sc = r4[16];
#pragma unroll
    for (int w = 1; w < NT / 128; ++w) {
        const float4 x = r4[w], y = r4[8 + w], z = r4[16 + w];
        sa = make_float4(sa.x + x.x, sa.y + x.y, sa.z + x.z, sa.w + x.w);
        sb = make_float4(sb.x + y.x, sb.y + y.y, sb.z + y.z, sb.w + y.w);
        sc = make_float4(sc.x + z.x, sc.y + z.y, sc.z + z.z, sc.w + z.w);
    }
    a = (sa.x + sa.y) + (sa.z + sa.w);
    b = (sb.x + sb.y) + (sb.z + sb.w);
    c = (sc.x + sc.y) + (sc.z + sc.w);
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

template <int MODE, class SP, class GA, class CL>
__global__ void __launch_bounds__(256) k_sap_colour(Geom g, SP b, SP x, GA U, CL C, CL Ci, typename SP::Real kappa,
                                                    int colour, int nmr, int x_zero)
{
    using T = typename SP::Real;
    extern __shared__ __align__(128) unsigned char smem[];
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

    // 1. block residual (of D, or of A = C^-1 D with C holding C^-1)
    Cx<T> rv[12];
    bb.load(i, rv);
    if (!x_zero) {
        if (MODE == SAP_JAC) {
            Cx<T> acc[12], t[12], xo[12];
            hop_site<false>(g, c, i, xx, U, acc);
            clover_site(C, i, acc, t);
            xx.load(i, xo);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<T>{fma(kappa, t[k].r, rv[k].r - xo[k].r), fma(kappa, t[k].i, rv[k].i - xo[k].i)};
        } else {
            Cx<T> dx[12];
            dirac_site<false>(g, c, i, xx, U, C, kappa, dx);
#pragma unroll
            for (int k = 0; k < 12; ++k) rv[k] = rv[k] - dx[k];
        }
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

    // 2''. even-odd preconditioned MR
    if (MODE == SAP_EO) {
        const bool even = l < (vb >> 1);
        Cx<T> rho[12], t[12], acc[12];
        auto hops = [&]() {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = Cx<T>{0, 0};
            block_hop_dir<0>(U, blkbase, i, nf[0], nb[0], rs, vb, acc);
            block_hop_dir<1>(U, blkbase, i, nf[1], nb[1], rs, vb, acc);
            block_hop_dir<2>(U, blkbase, i, nf[2], nb[2], rs, vb, acc);
            block_hop_dir<3>(U, blkbase, i, nf[3], nb[3], rs, vb, acc);
        };
        // rho = r_e + kappa H_eo C_oo^-1 r_o
        if (!even) {
            clover_site(Ci, i, rv, t);
#pragma unroll
            for (int k = 0; k < 12; ++k) rs[k * vb + l] = t[k];
        }
        __syncthreads();
        if (even) {
            hops();
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rho[k] = Cx<T>{fma(kappa, acc[k].r, rv[k].r), fma(kappa, acc[k].i, rv[k].i)};
        }
        __syncthreads();
        if (even)
#pragma unroll
            for (int k = 0; k < 12; ++k) rs[k * vb + l] = rho[k];
        __syncthreads();
        for (int it = 0; it < nmr; ++it) {
            // odd sites: y = C_oo^-1 (kappa H_oe rho)
            if (!even) {
                hops();
#pragma unroll
                for (int k = 0; k < 12; ++k) acc[k] = kappa * acc[k];
                clover_site(Ci, i, acc, t);
#pragma unroll
                for (int k = 0; k < 12; ++k) rs[k * vb + l] = t[k];
            }
            __syncthreads();
            // even sites: p = C_ee rho - kappa H_eo y, MR step
            T pr = 0, pi = 0, pp = 0;
            Cx<T> p[12];
            if (even) {
                hops();
                clover_site(C, i, rho, p);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    p[k] = Cx<T>{fma(-kappa, acc[k].r, p[k].r), fma(-kappa, acc[k].i, p[k].i)};
                    pr = fma(p[k].r, rho[k].r, fma(p[k].i, rho[k].i, pr));
                    pi = fma(p[k].r, rho[k].i, fma(-p[k].i, rho[k].r, pi));
                    pp = fma(p[k].r, p[k].r, fma(p[k].i, p[k].i, pp));
                }
            }
            block_sum3(pr, pi, pp, red);
            const Cx<T> alpha = (pp > 0) ? Cx<T>{pr / pp, pi / pp} : Cx<T>{0, 0};
            if (even)
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    e[k] = cfma(alpha, rho[k], e[k]);
                    rho[k] = rho[k] - alpha * p[k];
                    rs[k * vb + l] = rho[k];
                }
            __syncthreads();
        }
        // e_o = C_oo^-1 (r_o + kappa H_oe e_e)
        if (even)
#pragma unroll
            for (int k = 0; k < 12; ++k) rs[k * vb + l] = e[k];
        __syncthreads();
        if (!even) {
            hops();
#pragma unroll
            for (int k = 0; k < 12; ++k)
                t[k] = Cx<T>{fma(kappa, acc[k].r, rv[k].r), fma(kappa, acc[k].i, rv[k].i)};
            clover_site(Ci, i, t, e);
        }
        nmr = 0;
    }

    // 2'. Jacobi on A_B: e_1 = r_B, then e <- r_B + kappa C^-1 H_B e
    if (MODE == SAP_JAC) {
        if (nmr >= 1)
#pragma unroll
            for (int k = 0; k < 12; ++k) e[k] = rv[k];
        for (int it = 1; it < nmr; ++it) {
            Cx<T> acc[12], t[12];
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = Cx<T>{0, 0};
            block_hop_dir<0>(U, blkbase, i, nf[0], nb[0], rs, vb, acc);
            block_hop_dir<1>(U, blkbase, i, nf[1], nb[1], rs, vb, acc);
            block_hop_dir<2>(U, blkbase, i, nf[2], nb[2], rs, vb, acc);
            block_hop_dir<3>(U, blkbase, i, nf[3], nb[3], rs, vb, acc);
            clover_site(C, i, acc, t);
            __syncthreads();  // every thread has read e before it is replaced
#pragma unroll
            for (int k = 0; k < 12; ++k) {
                e[k] = Cx<T>{fma(kappa, t[k].r, rv[k].r), fma(kappa, t[k].i, rv[k].i)};
                rs[k * vb + l] = e[k];
            }
            __syncthreads();
        }
        nmr = 0;
    }

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

// ------------------------------------------------------------------ staged kernel
// The FP32/FP16-storage smoother keeps one domain's links and clover term in
// shared memory for the whole domain solve.  In the packed layout they are
// contiguous per domain, so one thread issues 1-D TMA bulk copies for them
// (completed on an mbarrier) while the block computes the hopping part of the
// domain residual from global memory.  r and e of the MR iteration also live in
// shared memory, which keeps the kernel at two resident blocks per SM.

// shared-memory views of one domain's links: the global plane layout with the
// domain index dropped (site index l inside the domain)
template <class GA> struct Staged;
template <> struct Staged<Gauge16x12> {
    static constexpr int BYTES = 96;  // per site, four links
    const uint2 *s;
    int lvb;
    static __device__ const void *src(const Gauge16x12 &U, int blk) { return U.p + ((size_t)blk * 12 << U.lvb); }
    __device__ __forceinline__ void load(int l, int mu, Cx<float> u[9]) const
    {
        const uint2 *q = s + ((mu * 3) << lvb) + l;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const uint2 v = q[k << lvb];
            const float2 a = unpack_half2(v.x), b = unpack_half2(v.y);
            u[2 * k] = {a.x, a.y};
            u[2 * k + 1] = {b.x, b.y};
        }
        reconstruct_row2(u);
    }
};
template <> struct Staged<Gauge16x18> {
    static constexpr int BYTES = 144;
    const uint32_t *s;
    int lvb;
    static __device__ const void *src(const Gauge16x18 &U, int blk) { return U.p + ((size_t)blk * 36 << U.lvb); }
    __device__ __forceinline__ void load(int l, int mu, Cx<float> u[9]) const
    {
        const uint32_t *q = s + ((mu * 9) << lvb) + l;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 a = unpack_half2(q[k << lvb]);
            u[k] = {a.x, a.y};
        }
    }
};
template <> struct Staged<Gauge32x12> {
    static constexpr int BYTES = 192;
    const float4 *s;
    int lvb;
    static __device__ const void *src(const Gauge32x12 &U, int blk) { return U.p + ((size_t)blk * 12 << U.lvb); }
    __device__ __forceinline__ void load(int l, int mu, Cx<float> u[9]) const
    {
        const float4 *q = s + ((mu * 3) << lvb) + l;
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            const float4 v = q[k << lvb];
            u[2 * k] = {v.x, v.y};
            u[2 * k + 1] = {v.z, v.w};
        }
        reconstruct_row2(u);
    }
};
template <> struct Staged<Gauge32x18> {
    static constexpr int BYTES = 288;
    const float2 *s;
    int lvb;
    static __device__ const void *src(const Gauge32x18 &U, int blk) { return U.p + ((size_t)blk * 36 << U.lvb); }
    __device__ __forceinline__ void load(int l, int mu, Cx<float> u[9]) const
    {
        const float2 *q = s + ((mu * 9) << lvb) + l;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const float2 v = q[k << lvb];
            u[k] = {v.x, v.y};
        }
    }
};

// the clover term of one domain in shared memory; mul() applies it to a site
template <class CL> struct StagedC;
template <> struct StagedC<Clover16> {
    static constexpr int BYTES = 144, SCALE = 4;
    const uint4 *s;
    const float *sc;
    int lvb;
    static __device__ const void *src(const Clover16 &C, int blk) { return C.p + ((size_t)blk * 9 << C.lvb); }
    static __device__ const void *src_scale(const Clover16 &C, int blk) { return C.sc + ((size_t)blk << C.lvb); }
    // the 72 halves pair up as (diagonal, diagonal) and (re, im) of the
    // off-diagonal entries: 18 packed words per chiral block
    __device__ __forceinline__ void mul(int l, const Cx<float> in[12], Cx<float> out[12]) const
    {
        uint32_t w[36];
        const uint4 *q = s + l;
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            const uint4 v = q[k << lvb];
            w[4 * k] = v.x;
            w[4 * k + 1] = v.y;
            w[4 * k + 2] = v.z;
            w[4 * k + 3] = v.w;
        }
        const float scale = sc[l];
#pragma unroll
        for (int chi = 0; chi < 2; ++chi) {
            const uint32_t *b = w + 18 * chi;
            const Cx<float> *v = in + 6 * chi;
            Cx<float> *o = out + 6 * chi;
#pragma unroll
            for (int a = 0; a < 3; ++a) {
                const float2 d = unpack_half2(b[a]);
                o[2 * a] = d.x * v[2 * a];
                o[2 * a + 1] = d.y * v[2 * a + 1];
            }
            int k = 3;
#pragma unroll
            for (int a = 1; a < 6; ++a)
#pragma unroll
                for (int c = 0; c < a; ++c) {
                    const float2 L = unpack_half2(b[k++]);
                    const Cx<float> Lc = {L.x, L.y};
                    o[a] = cfma(Lc, v[c], o[a]);
                    o[c] = cjfma(Lc, v[a], o[c]);
                }
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) out[k] = scale * out[k];
    }
};
template <> struct StagedC<Clover32> {
    static constexpr int BYTES = 288, SCALE = 0;
    const float4 *s;
    const float *sc;
    int lvb;
    static __device__ const void *src(const Clover32 &C, int blk) { return C.p + ((size_t)blk * 18 << C.lvb); }
    static __device__ const void *src_scale(const Clover32 &, int) { return nullptr; }
    __device__ __forceinline__ void mul(int l, const Cx<float> in[12], Cx<float> out[12]) const
    {
        float c[72];
        const float4 *q = s + l;
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            const float4 v = q[k << lvb];
            c[4 * k] = v.x;
            c[4 * k + 1] = v.y;
            c[4 * k + 2] = v.z;
            c[4 * k + 3] = v.w;
        }
        clover_mul(c, in, out);
    }
};

template <int MU, class SL>
__device__ __forceinline__ void staged_hop_dir(const SL &U, int l, int nf, int nb, const Cx<float> *rs, int vb,
                                               Cx<float> acc[12])
{
    Cx<float> s[12], h[6], w[6], u[9];
    if (nf >= 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = rs[k * vb + nf];
        project<MU, -1>(s, h);
        U.load(l, MU, u);
        su3_mul(u, h, w);
        reconstruct_add<MU, -1>(acc, w);
    }
    if (nb >= 0) {
#pragma unroll
        for (int k = 0; k < 12; ++k) s[k] = rs[k * vb + nb];
        project<MU, +1>(s, h);
        U.load(nb, MU, u);
        su3_dag_mul(u, h, w);
        reconstruct_add<MU, +1>(acc, w);
    }
}

// shared-memory bytes of the staged kernel for a domain of vb sites
// thread blocks of 256 threads per SM the staged kernel's shared memory allows
// (2 only for FP16 storage with 12-real links); the register bound follows
template <class GA, class CL>
__host__ __device__ constexpr int staged_min_ctas()
{
    return 2 * (256 * (Staged<GA>::BYTES + StagedC<CL>::BYTES + StagedC<CL>::SCALE + 2 * 12 * 8) + 400 + 1024) <=
                   228 * 1024
               ? 2
               : 1;
}

template <class GA, class CL>
static size_t staged_smem(int vb)
{
    return (size_t)vb * (Staged<GA>::BYTES + StagedC<CL>::BYTES + StagedC<CL>::SCALE + 2 * 12 * sizeof(Cx<float>)) +
           96 * sizeof(float) + 16;
}

// one domain solve of the staged kernel: domain jb of `colour`, right-hand side rr
template <int MODE, class SP, class GA, class CL>
__device__ __forceinline__ void sap_staged_body(const Geom &g, const SP &b, const SP &x, const GA &U, const CL &C,
                                                const CL &Ci, float kappa, int colour, int nmr, int x_zero,
                                                int *status, int jb, int rr);

// the even-odd solver keeps more state per thread: one block per SM
template <int MODE, class SP, class GA, class CL>
__global__ void __launch_bounds__(256, MODE == SAP_EO ? 1 : staged_min_ctas<GA, CL>())
    k_sap_staged(Geom g, SP b, SP x, GA U, CL C, CL Ci, float kappa, int colour, int nmr, int x_zero, int *status)
{
    sap_staged_body<MODE>(g, b, x, U, C, Ci, kappa, colour, nmr, x_zero, status, blockIdx.x, blockIdx.y);
}

template <int MODE, class SP, class GA, class CL>
__device__ __forceinline__ void sap_staged_body(const Geom &g, const SP &b, const SP &x, const GA &U, const CL &C,
                                                const CL &Ci, float kappa, int colour, int nmr, int x_zero,
                                                int *status, int jb, int rr)
{
    using SL = Staged<GA>;
    using SC = StagedC<CL>;
    extern __shared__ __align__(128) unsigned char smem[];
    const int vb = 1 << g.lvb;
    unsigned char *sp = smem;
    void *s_links = sp;
    sp += (size_t)SL::BYTES * vb;
    void *s_clov = sp;
    sp += (size_t)SC::BYTES * vb;
    float *s_scale = reinterpret_cast<float *>(sp);
    sp += (size_t)SC::SCALE * vb;
    Cx<float> *rs = reinterpret_cast<Cx<float> *>(sp);
    sp += (size_t)12 * vb * sizeof(Cx<float>);
    Cx<float> *es = reinterpret_cast<Cx<float> *>(sp);
    sp += (size_t)12 * vb * sizeof(Cx<float>);
    float *red = reinterpret_cast<float *>(sp);
    sp += 96 * sizeof(float);
    uint64_t *bar = reinterpret_cast<uint64_t *>(sp);

    const SP bb = shift_rhs(b, rr, g.V);
    const SP xx = shift_rhs(x, rr, g.V);
    int j = jb;
    const int half0 = g.NB[0] >> 1;
    int bc[4];
    const int m = j % half0;
    j /= half0;
    bc[1] = j % g.NB[1];
    j /= g.NB[1];
    bc[2] = j % g.NB[2];
    bc[3] = j / g.NB[2];
    bc[0] = 2 * m + ((colour + bc[1] + bc[2] + bc[3]) & 1);
    const int blk = block_index(g, bc);
    const int l = threadIdx.x;
    const int i = (blk << g.lvb) | l;

    // stage the domain's links and clover term
    if (l == 0) mbar_init(bar, 1);
    __syncthreads();
    if (l == 0) {
        const unsigned lb = SL::BYTES * vb, cb = SC::BYTES * vb, sb = SC::SCALE * vb;
        mbar_arrive_expect_tx(bar, lb + cb + sb);
        bulk_g2s(s_links, SL::src(U, blk), lb, bar);
        bulk_g2s(s_clov, SC::src(C, blk), cb, bar);
        if (SC::SCALE) bulk_g2s(s_scale, SC::src_scale(C, blk), sb, bar);
    }
    const SL Us{reinterpret_cast<decltype(SL::s)>(s_links), g.lvb};
    const SC Cs{reinterpret_cast<decltype(SC::s)>(s_clov), s_scale, g.lvb};

    int lc[4], c[4];
    local_coords(g, l, lc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) c[mu] = (bc[mu] << g.lb[mu]) + lc[mu];

    // 1. the hopping part of D x from global memory while the copies land
    Cx<float> acc[12], xs[12];
    if (!x_zero) hop_site<false>(g, c, i, xx, U, acc);

    const bool ok = mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
    if (!__syncthreads_and(ok)) {
        // give the copies in flight a second bounded chance, then report
        mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
        if (l == 0) atomicOr(status, MGC_DEV_TIMEOUT);
        return;
    }

    Cx<float> rv[12];
    bb.load(i, rv);
    if (!x_zero) {
        Cx<float> cx[12];
        xx.load(i, xs);
        if (MODE == SAP_JAC) {
            Cs.mul(l, acc, cx);  // C^-1 H x
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<float>{fmaf(kappa, cx[k].r, rv[k].r - xs[k].r), fmaf(kappa, cx[k].i, rv[k].i - xs[k].i)};
        } else {
            Cs.mul(l, xs, cx);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<float>{rv[k].r - fmaf(-kappa, acc[k].r, cx[k].r),
                                  rv[k].i - fmaf(-kappa, acc[k].i, cx[k].i)};
        }
    }
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
    for (int k = 0; k < 12; ++k) {
        rs[k * vb + l] = rv[k];
        es[k * vb + l] = Cx<float>{0.f, 0.f};
    }
    __syncthreads();

    // 2''. even-odd preconditioned MR (C^-1 of the odd sites from global memory)
    if (MODE == SAP_EO) {
        const bool even = l < (vb >> 1);
        Cx<float> rho[12], t[12], ee[12];
        auto hops = [&]() {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = Cx<float>{0.f, 0.f};
            staged_hop_dir<0>(Us, l, nf[0], nb[0], rs, vb, acc);
            staged_hop_dir<1>(Us, l, nf[1], nb[1], rs, vb, acc);
            staged_hop_dir<2>(Us, l, nf[2], nb[2], rs, vb, acc);
            staged_hop_dir<3>(Us, l, nf[3], nb[3], rs, vb, acc);
        };
#pragma unroll
        for (int k = 0; k < 12; ++k) ee[k] = Cx<float>{0.f, 0.f};
        if (!even) {
            clover_site(Ci, i, rv, t);
#pragma unroll
            for (int k = 0; k < 12; ++k) rs[k * vb + l] = t[k];
        }
        __syncthreads();
        if (even) {
            hops();
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rho[k] = Cx<float>{fmaf(kappa, acc[k].r, rv[k].r), fmaf(kappa, acc[k].i, rv[k].i)};
        }
        __syncthreads();
        if (even)
#pragma unroll
            for (int k = 0; k < 12; ++k) rs[k * vb + l] = rho[k];
        __syncthreads();
        for (int it = 0; it < nmr; ++it) {
            if (!even) {
                hops();
#pragma unroll
                for (int k = 0; k < 12; ++k) acc[k] = kappa * acc[k];
                clover_site(Ci, i, acc, t);
#pragma unroll
                for (int k = 0; k < 12; ++k) rs[k * vb + l] = t[k];
            }
            __syncthreads();
            float pr = 0.f, pi = 0.f, pp = 0.f;
            Cx<float> p[12];
            if (even) {
                hops();
                Cs.mul(l, rho, p);
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    p[k] = Cx<float>{fmaf(-kappa, acc[k].r, p[k].r), fmaf(-kappa, acc[k].i, p[k].i)};
                    pr = fmaf(p[k].r, rho[k].r, fmaf(p[k].i, rho[k].i, pr));
                    pi = fmaf(p[k].r, rho[k].i, fmaf(-p[k].i, rho[k].r, pi));
                    pp = fmaf(p[k].r, p[k].r, fmaf(p[k].i, p[k].i, pp));
                }
            }
            block_sum3(pr, pi, pp, red);
            const Cx<float> alpha = (pp > 0.f) ? Cx<float>{pr / pp, pi / pp} : Cx<float>{0.f, 0.f};
            if (even)
#pragma unroll
                for (int k = 0; k < 12; ++k) {
                    ee[k] = cfma(alpha, rho[k], ee[k]);
                    rho[k] = rho[k] - alpha * p[k];
                    rs[k * vb + l] = rho[k];
                }
            __syncthreads();
        }
        if (even)
#pragma unroll
            for (int k = 0; k < 12; ++k) rs[k * vb + l] = ee[k];
        __syncthreads();
        if (!even) {
            hops();
#pragma unroll
            for (int k = 0; k < 12; ++k)
                t[k] = Cx<float>{fmaf(kappa, acc[k].r, rv[k].r), fmaf(kappa, acc[k].i, rv[k].i)};
            clover_site(Ci, i, t, ee);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) es[k * vb + l] = ee[k];
        nmr = 0;
    }

    // 2'. Jacobi on A_B with e in shared memory (rs): e_1 = r_B, then
    // e <- r_B + kappa C^-1 H_B e
    if (MODE == SAP_JAC) {
        for (int it = 1; it < nmr; ++it) {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = Cx<float>{0.f, 0.f};
            staged_hop_dir<0>(Us, l, nf[0], nb[0], rs, vb, acc);
            staged_hop_dir<1>(Us, l, nf[1], nb[1], rs, vb, acc);
            staged_hop_dir<2>(Us, l, nf[2], nb[2], rs, vb, acc);
            staged_hop_dir<3>(Us, l, nf[3], nb[3], rs, vb, acc);
            Cx<float> t[12];
            Cs.mul(l, acc, t);
            __syncthreads();  // every thread has read e before it is replaced
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rs[k * vb + l] = Cx<float>{fmaf(kappa, t[k].r, rv[k].r), fmaf(kappa, t[k].i, rv[k].i)};
            __syncthreads();
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) es[k * vb + l] = nmr >= 1 ? rs[k * vb + l] : Cx<float>{0.f, 0.f};
        nmr = 0;
    }

    // 2. minimal residual on D_B with links, clover and r in shared memory
    for (int it = 0; it < nmr; ++it) {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = Cx<float>{0.f, 0.f};
        staged_hop_dir<0>(Us, l, nf[0], nb[0], rs, vb, acc);
        staged_hop_dir<1>(Us, l, nf[1], nb[1], rs, vb, acc);
        staged_hop_dir<2>(Us, l, nf[2], nb[2], rs, vb, acc);
        staged_hop_dir<3>(Us, l, nf[3], nb[3], rs, vb, acc);
        Cx<float> p[12];
        Cs.mul(l, rv, p);
        float pr = 0.f, pi = 0.f, pp = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k] = Cx<float>{fmaf(-kappa, acc[k].r, p[k].r), fmaf(-kappa, acc[k].i, p[k].i)};
            pr = fmaf(p[k].r, rv[k].r, fmaf(p[k].i, rv[k].i, pr));
            pi = fmaf(p[k].r, rv[k].i, fmaf(-p[k].i, rv[k].r, pi));
            pp = fmaf(p[k].r, p[k].r, fmaf(p[k].i, p[k].i, pp));
        }
        block_sum3(pr, pi, pp, red);
        const Cx<float> alpha = (pp > 0.f) ? Cx<float>{pr / pp, pi / pp} : Cx<float>{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            es[k * vb + l] = cfma(alpha, rv[k], es[k * vb + l]);
            rv[k] = rv[k] - alpha * p[k];
            rs[k * vb + l] = rv[k];
        }
        __syncthreads();
    }

    // 3. x_B += e
    Cx<float> e[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = es[k * vb + l];
    if (!x_zero) {
#pragma unroll
        for (int k = 0; k < 12; ++k) e[k] = e[k] + xs[k];
    }
    xx.store(i, e);
}

// ------------------------------------------------------------------ FP16-storage kernel
// The benchmark format (FP16 fields with per-site scales) for 2^4 and 4^4
// domains, with the domain size known at compile time.  Shared memory holds
// the domain's links as 18-real FP16 (a 12-real copy is brought in by TMA into
// the r area and expanded once, so the MR steps never rebuild row 2), the FP16
// clover term with its scales, and r as pairs of complex numbers.  e stays in
// registers; a thread re-reads its own r from shared memory when it needs it.
// About 100 KB of shared memory: two blocks per SM.

template <class GA> struct H16Links;
template <> struct H16Links<Gauge16x12> {
    static constexpr bool EXPAND = true;
    static constexpr int STAGE = 96;  // bytes per site of the staged copy
    static __device__ const void *src(const Gauge16x12 &U, int blk, int lvb) { return U.p + ((size_t)blk * 12 << lvb); }
};
template <> struct H16Links<Gauge16x18> {
    static constexpr bool EXPAND = false;
    static constexpr int STAGE = 144;
    static __device__ const void *src(const Gauge16x18 &U, int blk, int lvb) { return U.p + ((size_t)blk * 36 << lvb); }
};

template <int LVB>
__host__ __device__ constexpr size_t h16_smem_bytes()
{
    return (size_t)(1 << LVB) * (144 + 144 + 4 + 96) + 96 * 4 + 16;
}

template <int MU, int SGN, int VB>
__device__ __forceinline__ void h16_hop(const float4 *rs, int n, const uint32_t *sL, int lk, Cx<float> acc[12])
{
    Cx<float> s[12], h[6], w[6], u[9];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 v = rs[k * VB + n];
        s[2 * k] = {v.x, v.y};
        s[2 * k + 1] = {v.z, v.w};
    }
    project<MU, SGN>(s, h);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float2 v = unpack_half2(sL[(MU * 9 + k) * VB + lk]);
        u[k] = {v.x, v.y};
    }
    if (SGN < 0) su3_mul(u, h, w);
    else su3_dag_mul(u, h, w);
    reconstruct_add<MU, SGN>(acc, w);
}

// one domain solve of the FP16 kernel: domain jb of `colour`, right-hand side rr
template <bool JAC, int LVB, class GA>
__device__ __forceinline__ void sap_h16_body(const Geom &g, const Spinor16 &b, const Spinor16 &x, const GA &U,
                                             const Clover16 &C, float kappa, int colour, int nmr, int x_zero,
                                             int *status, int jb, int rr);

template <bool JAC, int LVB, class GA>
__global__ void __launch_bounds__(1 << LVB, 2) k_sap_h16(Geom g, Spinor16 b, Spinor16 x, GA U, Clover16 C, float kappa,
                                                         int colour, int nmr, int x_zero, int *status)
{
    sap_h16_body<JAC, LVB>(g, b, x, U, C, kappa, colour, nmr, x_zero, status, blockIdx.x, blockIdx.y);
}

template <bool JAC, int LVB, class GA>
__device__ __forceinline__ void sap_h16_body(const Geom &g, const Spinor16 &b, const Spinor16 &x, const GA &U,
                                             const Clover16 &C, float kappa, int colour, int nmr, int x_zero,
                                             int *status, int jb, int rr)
{
    constexpr int VB = 1 << LVB;
    constexpr int LB = LVB / 4;
    using HL = H16Links<GA>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t *sL = reinterpret_cast<uint32_t *>(smem);        // [4][9][VB] half2
    uint4 *sC = reinterpret_cast<uint4 *>(sL + 36 * VB);      // [9][VB]
    float *sS = reinterpret_cast<float *>(sC + 9 * VB);       // [VB]
    float4 *rs = reinterpret_cast<float4 *>(sS + VB);         // [6][VB]; first the 12-real link stage
    float *red = reinterpret_cast<float *>(rs + 6 * VB);      // 96 floats
    uint64_t *bar = reinterpret_cast<uint64_t *>(red + 96);

    // geometry with the domain extents as compile-time constants
    Geom gg = g;
    gg.lvb = LVB;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LB;
    Spinor16 bb = shift_rhs(b, rr, g.V), xx = shift_rhs(x, rr, g.V);
    bb.lvb = LVB;
    xx.lvb = LVB;
    GA Ug = U;
    Ug.lvb = LVB;
    int j = jb;
    const int half0 = g.NB[0] >> 1;
    int bc[4];
    const int m = j % half0;
    j /= half0;
    bc[1] = j % g.NB[1];
    j /= g.NB[1];
    bc[2] = j % g.NB[2];
    bc[3] = j / g.NB[2];
    bc[0] = 2 * m + ((colour + bc[1] + bc[2] + bc[3]) & 1);
    const int blk = block_index(gg, bc);
    const int l = threadIdx.x;
    const int i = (blk << LVB) | l;

    if (l == 0) mbar_init(bar, 1);
    __syncthreads();
    static_assert(HL::STAGE * VB % 16 == 0 && 144 * VB % 16 == 0 && 4 * VB % 16 == 0,
                  "bulk copies move multiples of 16 bytes");
    if (l == 0) {
        const unsigned lbytes = HL::STAGE * VB, cb = 144 * VB, sb = 4 * VB;
        mbar_arrive_expect_tx(bar, lbytes + cb + sb);
        bulk_g2s(HL::EXPAND ? (void *)rs : (void *)sL, HL::src(U, blk, LVB), lbytes, bar);
        bulk_g2s(sC, C.p + ((size_t)blk * 9 << LVB), cb, bar);
        bulk_g2s(sS, C.sc + ((size_t)blk << LVB), sb, bar);
    }
    // a programmatic dependent of the previous colour launch (as in the MR
    // kernel): x is read only once that launch has completed
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    int lc[4], cg[4];
    local_coords(gg, l, lc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) cg[mu] = (bc[mu] << LB) + lc[mu];

    // 1. hopping part of D x from global memory while the copies land
    Cx<float> acc[12];
    if (!x_zero) hop_site<false>(gg, cg, i, xx, Ug, acc);

    const bool ok = mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
    if (!__syncthreads_and(ok)) {
        mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
        if (l == 0) atomicOr(status, MGC_DEV_TIMEOUT);
        return;
    }
    if (HL::EXPAND) {
        // rows 0 and 1 staged in the r area; row 2 = conj(row0 x row1) once per link
        const uint2 *st = reinterpret_cast<const uint2 *>(rs);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            Cx<float> u[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint2 v = st[(mu * 3 + k) * VB + l];
                const float2 a = unpack_half2(v.x), c2 = unpack_half2(v.y);
                u[2 * k] = {a.x, a.y};
                u[2 * k + 1] = {c2.x, c2.y};
            }
            reconstruct_row2(u);
#pragma unroll
            for (int k = 0; k < 9; ++k) sL[(mu * 9 + k) * VB + l] = pack_half2(u[k].r, u[k].i);
        }
        __syncthreads();  // links complete, r area free
    }
    const StagedC<Clover16> Cs{sC, sS, LVB};

    Cx<float> rv[12];
    bb.load(i, rv);
    if (!x_zero) {
        Cx<float> xs[12], cx[12];
        xx.load(i, xs);
        if (JAC) {
            Cs.mul(l, acc, cx);  // C^-1 H x
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<float>{fmaf(kappa, cx[k].r, rv[k].r - xs[k].r), fmaf(kappa, cx[k].i, rv[k].i - xs[k].i)};
        } else {
            Cs.mul(l, xs, cx);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<float>{rv[k].r - fmaf(-kappa, acc[k].r, cx[k].r),
                                  rv[k].i - fmaf(-kappa, acc[k].i, cx[k].i)};
        }
    }
    int nf[4], nb[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int t[4] = {lc[0], lc[1], lc[2], lc[3]};
        t[mu] = lc[mu] + 1;
        nf[mu] = (t[mu] < (1 << LB)) ? local_index(gg, t) : -1;
        t[mu] = lc[mu] - 1;
        nb[mu] = (t[mu] >= 0) ? local_index(gg, t) : -1;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) rs[k * VB + l] = make_float4(rv[2 * k].r, rv[2 * k].i, rv[2 * k + 1].r, rv[2 * k + 1].i);
    Cx<float> e[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = Cx<float>{0.f, 0.f};
    __syncthreads();

    // 2'. Jacobi on A_B with e in shared memory (rs): e_1 = r_B, then
    // e <- r_B + kappa C^-1 H_B e
    if (JAC) {
        if (nmr >= 1)
#pragma unroll
            for (int k = 0; k < 12; ++k) e[k] = rv[k];
        for (int it = 1; it < nmr; ++it) {
#pragma unroll
            for (int k = 0; k < 12; ++k) acc[k] = Cx<float>{0.f, 0.f};
            if (nf[0] >= 0) h16_hop<0, -1, VB>(rs, nf[0], sL, l, acc);
            if (nb[0] >= 0) h16_hop<0, +1, VB>(rs, nb[0], sL, nb[0], acc);
            if (nf[1] >= 0) h16_hop<1, -1, VB>(rs, nf[1], sL, l, acc);
            if (nb[1] >= 0) h16_hop<1, +1, VB>(rs, nb[1], sL, nb[1], acc);
            if (nf[2] >= 0) h16_hop<2, -1, VB>(rs, nf[2], sL, l, acc);
            if (nb[2] >= 0) h16_hop<2, +1, VB>(rs, nb[2], sL, nb[2], acc);
            if (nf[3] >= 0) h16_hop<3, -1, VB>(rs, nf[3], sL, l, acc);
            if (nb[3] >= 0) h16_hop<3, +1, VB>(rs, nb[3], sL, nb[3], acc);
            Cx<float> t[12];
            Cs.mul(l, acc, t);
            __syncthreads();  // every thread has read e before it is replaced
#pragma unroll
            for (int k = 0; k < 12; ++k) e[k] = Cx<float>{fmaf(kappa, t[k].r, rv[k].r), fmaf(kappa, t[k].i, rv[k].i)};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                rs[k * VB + l] = make_float4(e[2 * k].r, e[2 * k].i, e[2 * k + 1].r, e[2 * k + 1].i);
            __syncthreads();
        }
        nmr = 0;
    }

    // 2. minimal residual on D_B
    for (int it = 0; it < nmr; ++it) {
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[k] = Cx<float>{0.f, 0.f};
        if (nf[0] >= 0) h16_hop<0, -1, VB>(rs, nf[0], sL, l, acc);
        if (nb[0] >= 0) h16_hop<0, +1, VB>(rs, nb[0], sL, nb[0], acc);
        if (nf[1] >= 0) h16_hop<1, -1, VB>(rs, nf[1], sL, l, acc);
        if (nb[1] >= 0) h16_hop<1, +1, VB>(rs, nb[1], sL, nb[1], acc);
        if (nf[2] >= 0) h16_hop<2, -1, VB>(rs, nf[2], sL, l, acc);
        if (nb[2] >= 0) h16_hop<2, +1, VB>(rs, nb[2], sL, nb[2], acc);
        if (nf[3] >= 0) h16_hop<3, -1, VB>(rs, nf[3], sL, l, acc);
        if (nb[3] >= 0) h16_hop<3, +1, VB>(rs, nb[3], sL, nb[3], acc);
        Cx<float> rv2[12], p[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = rs[k * VB + l];
            rv2[2 * k] = {v.x, v.y};
            rv2[2 * k + 1] = {v.z, v.w};
        }
        Cs.mul(l, rv2, p);
        float pr = 0.f, pi = 0.f, pp = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            p[k] = Cx<float>{fmaf(-kappa, acc[k].r, p[k].r), fmaf(-kappa, acc[k].i, p[k].i)};
            pr = fmaf(p[k].r, rv2[k].r, fmaf(p[k].i, rv2[k].i, pr));
            pi = fmaf(p[k].r, rv2[k].i, fmaf(-p[k].i, rv2[k].r, pi));
            pp = fmaf(p[k].r, p[k].r, fmaf(p[k].i, p[k].i, pp));
        }
        block_sum3(pr, pi, pp, red);
        const Cx<float> alpha = (pp > 0.f) ? Cx<float>{pr / pp, pi / pp} : Cx<float>{0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            e[k] = cfma(alpha, rv2[k], e[k]);
            rv2[k] = rv2[k] - alpha * p[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            rs[k * VB + l] = make_float4(rv2[2 * k].r, rv2[2 * k].i, rv2[2 * k + 1].r, rv2[2 * k + 1].i);
        __syncthreads();
    }

    // 3. x_B += e
    if (!x_zero) {
        Cx<float> xo[12];
        xx.load(i, xo);
#pragma unroll
        for (int k = 0; k < 12; ++k) e[k] = e[k] + xo[k];
    }
    xx.store(i, e);
}

// ---- the FP16 smoother's MR domain solve with FP16-operand arithmetic
// (hop16.cuh): the staged links and clover words and an FP16 copy of r (one
// FP32 scale per site, the storage convention of the FP16 fields) are the
// factors of D_B r, fed to the FP32 multiply-adds as stored.  r itself, e and
// p stay in FP32 registers: the inner products, alpha and the updates are the
// FP32 arithmetic of the MR step, and only the operator sees r rounded to
// FP16, as it sees every FP16-stored spinor.  Shared memory as in k_sap_h16,
// the r area holding the FP16 copy of r and its scales.

// The staged links of one domain in shared memory, as half2 words, entry k of
// link (lk, mu) at word k.  Links rebuilt from 12 reals in the kernel are
// stored packed ([4][2][VB] uint4 for words 0-7, then [4][VB] words 8), so a
// link takes three shared-memory loads; 18-real links keep their global
// layout ([4][9][VB] words), into which they are copied whole.
template <bool PACKED, int VB> struct SmemLinks16 {
    const uint32_t *w;
    template <int MU> __device__ __forceinline__ void load(int lk, uint32_t u[9]) const
    {
        if (PACKED) {
            const uint4 *w4 = reinterpret_cast<const uint4 *>(w);
            const uint4 a = w4[(MU * 2) * VB + lk], b = w4[(MU * 2 + 1) * VB + lk];
            u[0] = a.x; u[1] = a.y; u[2] = a.z; u[3] = a.w;
            u[4] = b.x; u[5] = b.y; u[6] = b.z; u[7] = b.w;
            u[8] = w[32 * VB + MU * VB + lk];
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) u[k] = w[(MU * 9 + k) * VB + lk];
        }
    }
    __device__ __forceinline__ void store(int mu, int l, const uint32_t u[9]) const
    {
        uint32_t *d = const_cast<uint32_t *>(w);
        if (PACKED) {
            uint4 *d4 = reinterpret_cast<uint4 *>(d);
            d4[(mu * 2) * VB + l] = make_uint4(u[0], u[1], u[2], u[3]);
            d4[(mu * 2 + 1) * VB + l] = make_uint4(u[4], u[5], u[6], u[7]);
            d[32 * VB + mu * VB + l] = u[8];
        } else {
#pragma unroll
            for (int k = 0; k < 9; ++k) d[(mu * 9 + k) * VB + l] = u[k];
        }
    }
};

template <int MU, int SGN, int VB, class SL>
__device__ __forceinline__ void m16_hop(const uint4 *r16, const float *rsc, int n, const SL &sL, int lk, float mk,
                                        float ar[12], float ai[12])
{
    uint32_t s[12], h[6], u[9];
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 v = r16[k * VB + n];
        s[4 * k] = v.x;
        s[4 * k + 1] = v.y;
        s[4 * k + 2] = v.z;
        s[4 * k + 3] = v.w;
    }
    const float coef = mk * rsc[n];
    project16<MU, SGN>(s, h);
    sL.template load<MU>(lk, u);
    float wr[6], wi[6];
    su3_mul16<(SGN > 0)>(u, h, wr, wi);
    reconstruct16<MU, SGN>(ar, ai, wr, wi, coef);
}

// r (FP32) to its FP16 copy at local site l: the site's largest |component| as
// the scale, components divided by it and rounded to nearest
template <int VB>
__device__ __forceinline__ void m16_store_r(uint4 *r16, float *rsc, int l, const float rr[12], const float ri[12])
{
    // the largest |component| by a tree of maxima
    float t[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) t[k] = fmaxf(fabsf(rr[k]), fabsf(ri[k]));
#pragma unroll
    for (int k = 0; k < 6; ++k) t[k] = fmaxf(t[k], t[k + 6]);
#pragma unroll
    for (int k = 0; k < 3; ++k) t[k] = fmaxf(t[k], t[k + 3]);
    const float m = fmaxf(fmaxf(t[0], t[1]), t[2]);
    // below FP32's normal range the site is stored as zero (1/m would overflow)
    const float inv = m >= FLT_MIN ? 1.0f / m : 0.f;
#pragma unroll
    for (int k = 0; k < 3; ++k)
        r16[k * VB + l] = make_uint4(pack_half2(rr[4 * k] * inv, ri[4 * k] * inv),
                                     pack_half2(rr[4 * k + 1] * inv, ri[4 * k + 1] * inv),
                                     pack_half2(rr[4 * k + 2] * inv, ri[4 * k + 2] * inv),
                                     pack_half2(rr[4 * k + 3] * inv, ri[4 * k + 3] * inv));
    rsc[l] = m;
}

template <int LVB, class GA>
__device__ __forceinline__ void sap_m16_body(const Geom &g, const Spinor16 &b, const Spinor16 &x, const GA &U,
                                             const Clover16 &C, float kappa, int colour, int nmr, int x_zero,
                                             int *status, int jb, int rr)
{
    constexpr int VB = 1 << LVB;
    constexpr int LB = LVB / 4;
    using HL = H16Links<GA>;
    extern __shared__ __align__(128) unsigned char smem[];
    uint32_t *sLw = reinterpret_cast<uint32_t *>(smem);    // 36 VB half2 words of links
    const SmemLinks16<HL::EXPAND, VB> sL{sLw};
    uint4 *sC = reinterpret_cast<uint4 *>(sLw + 36 * VB);  // [9][VB]
    float *sS = reinterpret_cast<float *>(sC + 9 * VB);    // [VB]
    uint4 *area = reinterpret_cast<uint4 *>(sS + VB);      // 96 VB bytes: 12-real link stage, then r
    uint4 *r16 = area;                                     // [3][VB] FP16 copy of r
    float *rsc = reinterpret_cast<float *>(area + 3 * VB); // [VB] its scales
    float *red = reinterpret_cast<float *>(area + 6 * VB); // 96 floats
    uint64_t *bar = reinterpret_cast<uint64_t *>(red + 96);
    static_assert(HL::STAGE * VB % 16 == 0 && 144 * VB % 16 == 0 && 4 * VB % 16 == 0,
                  "bulk copies move multiples of 16 bytes");
    static_assert(52 * VB <= 96 * VB, "the FP16 copy of r fits the stage area");

    Geom gg = g;
    gg.lvb = LVB;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LB;
    Spinor16 bb = shift_rhs(b, rr, g.V), xx = shift_rhs(x, rr, g.V);
    bb.lvb = LVB;
    xx.lvb = LVB;
    GA Ug = U;
    Ug.lvb = LVB;
    int j = jb;
    const int half0 = g.NB[0] >> 1;
    int bc[4];
    const int m = j % half0;
    j /= half0;
    bc[1] = j % g.NB[1];
    j /= g.NB[1];
    bc[2] = j % g.NB[2];
    bc[3] = j / g.NB[2];
    bc[0] = 2 * m + ((colour + bc[1] + bc[2] + bc[3]) & 1);
    const int blk = block_index(gg, bc);
    const int l = threadIdx.x;
    const int i = (blk << LVB) | l;

    if (l == 0) mbar_init(bar, 1);
    __syncthreads();
    if (l == 0) {
        const unsigned lbytes = HL::STAGE * VB, cb = 144 * VB, sb = 4 * VB;
        mbar_arrive_expect_tx(bar, lbytes + cb + sb);
        bulk_g2s(HL::EXPAND ? (void *)area : (void *)sLw, HL::src(U, blk, LVB), lbytes, bar);
        bulk_g2s(sC, C.p + ((size_t)blk * 9 << LVB), cb, bar);
        bulk_g2s(sS, C.sc + ((size_t)blk << LVB), sb, bar);
    }
    // launched as a programmatic dependent of the previous colour launch:
    // let the next launch take the SMs this one frees, and read x (written
    // by the previous launch) only once that launch has completed; the links
    // and clover copies above do not depend on it
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    int lc[4], cg[4];
    local_coords(gg, l, lc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) cg[mu] = (bc[mu] << LB) + lc[mu];

    // 1. hopping part of D x from global memory while the copies land
    float ar[12], ai[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) ar[k] = ai[k] = 0.f;
    if (!x_zero) {
        hop16_dir<0, false>(gg, cg, i, xx, Ug, -kappa, ar, ai);
        hop16_dir<1, false>(gg, cg, i, xx, Ug, -kappa, ar, ai);
        hop16_dir<2, false>(gg, cg, i, xx, Ug, -kappa, ar, ai);
        hop16_dir<3, false>(gg, cg, i, xx, Ug, -kappa, ar, ai);
    }

    const bool ok = mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
    if (!__syncthreads_and(ok)) {
        mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
        if (l == 0) atomicOr(status, MGC_DEV_TIMEOUT);
        return;
    }
    if (HL::EXPAND) {
        // rows 0 and 1 staged in the r area; row 2 = conj(row0 x row1) once per link
        const uint2 *st = reinterpret_cast<const uint2 *>(area);
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            uint32_t u[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint2 v = st[(mu * 3 + k) * VB + l];
                u[2 * k] = v.x;
                u[2 * k + 1] = v.y;
            }
            row2_16(u);
            sL.store(mu, l, u);
        }
        __syncthreads();  // links complete, r area free
    }

    // r_B = b - (C x - kappa H x)
    float rvr[12], rvi[12];
    {
        Cx<float> bv[12];
        bb.load(i, bv);
        if (!x_zero) {
            uint32_t v[12];
            words16(xx, i, v);
            clover_planes16<false>(sC + l, VB, v, sS[l] * xx.scale_of(i), ar, ai);
        }
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            rvr[k] = bv[k].r - ar[k];
            rvi[k] = bv[k].i - ai[k];
        }
    }
    int nf[4], nb[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int t[4] = {lc[0], lc[1], lc[2], lc[3]};
        t[mu] = lc[mu] + 1;
        nf[mu] = (t[mu] < (1 << LB)) ? local_index(gg, t) : -1;
        t[mu] = lc[mu] - 1;
        nb[mu] = (t[mu] >= 0) ? local_index(gg, t) : -1;
    }
    m16_store_r<VB>(r16, rsc, l, rvr, rvi);
    float er[12], ei[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) er[k] = ei[k] = 0.f;
    __syncthreads();

    // 2. minimal residual on D_B: p = D_B r (r's FP16 copy), alpha = <p, r>/<p, p>,
    // e += alpha r, r -= alpha p
    for (int it = 0; it < nmr; ++it) {
#pragma unroll
        for (int k = 0; k < 12; ++k) ar[k] = ai[k] = 0.f;
        {
            uint32_t v[12];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const uint4 w = r16[k * VB + l];
                v[4 * k] = w.x;
                v[4 * k + 1] = w.y;
                v[4 * k + 2] = w.z;
                v[4 * k + 3] = w.w;
            }
            clover_planes16<false>(sC + l, VB, v, sS[l] * rsc[l], ar, ai);
        }
        const float mk = -kappa;
        if (nf[0] >= 0) m16_hop<0, -1, VB>(r16, rsc, nf[0], sL, l, mk, ar, ai);
        if (nb[0] >= 0) m16_hop<0, +1, VB>(r16, rsc, nb[0], sL, nb[0], mk, ar, ai);
        if (nf[1] >= 0) m16_hop<1, -1, VB>(r16, rsc, nf[1], sL, l, mk, ar, ai);
        if (nb[1] >= 0) m16_hop<1, +1, VB>(r16, rsc, nb[1], sL, nb[1], mk, ar, ai);
        if (nf[2] >= 0) m16_hop<2, -1, VB>(r16, rsc, nf[2], sL, l, mk, ar, ai);
        if (nb[2] >= 0) m16_hop<2, +1, VB>(r16, rsc, nb[2], sL, nb[2], mk, ar, ai);
        if (nf[3] >= 0) m16_hop<3, -1, VB>(r16, rsc, nf[3], sL, l, mk, ar, ai);
        if (nb[3] >= 0) m16_hop<3, +1, VB>(r16, rsc, nb[3], sL, nb[3], mk, ar, ai);
        // <p, r> and <p, p> in four partial sums each (shorter dependent chains)
        float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f}, sp[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const int q = k & 3;
            sr[q] = fmaf(ar[k], rvr[k], fmaf(ai[k], rvi[k], sr[q]));
            si[q] = fmaf(ar[k], rvi[k], fmaf(-ai[k], rvr[k], si[q]));
            sp[q] = fmaf(ar[k], ar[k], fmaf(ai[k], ai[k], sp[q]));
        }
        float pr = (sr[0] + sr[1]) + (sr[2] + sr[3]);
        float pi = (si[0] + si[1]) + (si[2] + si[3]);
        float pp = (sp[0] + sp[1]) + (sp[2] + sp[3]);
        if constexpr (VB >= 128) block_sum3_v4<VB>(pr, pi, pp, red);
        else block_sum3(pr, pi, pp, red);
        // a domain whose <p, p> is below FP32's normal range takes no step
        // (1 / <p, p> would overflow)
        const float ipp = pp >= FLT_MIN ? 1.0f / pp : 0.f;
        const float alr = pr * ipp, ali = pi * ipp;
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            er[k] = fmaf(alr, rvr[k], fmaf(-ali, rvi[k], er[k]));
            ei[k] = fmaf(alr, rvi[k], fmaf(ali, rvr[k], ei[k]));
            rvr[k] = fmaf(-alr, ar[k], fmaf(ali, ai[k], rvr[k]));
            rvi[k] = fmaf(-alr, ai[k], fmaf(-ali, ar[k], rvi[k]));
        }
        m16_store_r<VB>(r16, rsc, l, rvr, rvi);
        __syncthreads();
    }

    // 3. x_B += e
    Cx<float> eo[12];
    if (!x_zero) {
        Cx<float> xo[12];
        xx.load(i, xo);
#pragma unroll
        for (int k = 0; k < 12; ++k) eo[k] = Cx<float>{er[k] + xo[k].r, ei[k] + xo[k].i};
    } else {
#pragma unroll
        for (int k = 0; k < 12; ++k) eo[k] = Cx<float>{er[k], ei[k]};
    }
    xx.store(i, eo);
}

template <int LVB, class GA>
__global__ void __launch_bounds__(1 << LVB, 2) k_sap_m16(Geom g, Spinor16 b, Spinor16 x, GA U, Clover16 C, float kappa,
                                                         int colour, int nmr, int x_zero, int *status)
{
    sap_m16_body<LVB>(g, b, x, U, C, kappa, colour, nmr, x_zero, status, blockIdx.x, blockIdx.y);
}

template <bool JAC, int LVB, class GA>
static int sap_run_h16(const mgc_clover_s *op, Spinor16 b, Spinor16 x, GA U, Clover16 C, int nrhs, int n_cy, int n_mr,
                       int x_is_zero, cudaStream_t s, int compress)
{
    const Geom &g = op->gauge->lat->g;
    constexpr size_t smem = h16_smem_bytes<LVB>();
    auto kern = JAC ? k_sap_h16<JAC, LVB, GA> : k_sap_m16<LVB, GA>;
    MGC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(g.nblocks / 2, nrhs);
    // colour launches after the first are programmatic dependents of the one
    // before (griddepcontrol in both kernels): their blocks start, and stage
    // their links and clover, while the previous launch's last blocks run
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(1 << LVB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    for (int cy = 0; cy < n_cy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int xz = (cy == 0 && colour == 0) ? x_is_zero : 0;
            if (cy > 0 || colour > 0)
                MGC_CUDA(cudaLaunchKernelEx(&cfg, kern, g, b, x, U, C, (float)op->kappa, colour, n_mr, xz,
                                            op->d_status));
            else
                kern<<<grid, 1 << LVB, smem, s>>>(g, b, x, U, C, (float)op->kappa, colour, n_mr, xz, op->d_status);
            count(1, sap_launch_bytes(g, 16, compress, nrhs, xz != 0));
        }
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

// ------------------------------------------------------------------ FP32-storage kernel
// FP32 fields on 2^4 and 4^4 domains with the domain size known at compile
// time.  Shared memory holds the domain's links as 18-real FP32 (a 12-real
// copy is brought in by TMA into the upper two thirds of that area and
// expanded once) and r as pairs of complex numbers; e stays in registers and
// the clover term is read from global memory at each use (it stays in L2
// across the MR steps).  About 98 KB of shared memory: two blocks per SM,
// where keeping the clover term in shared memory as well allows one.

template <class GA> struct F32Links;
template <> struct F32Links<Gauge32x12> {
    static constexpr bool EXPAND = true;
    static constexpr int STAGE = 192;  // bytes per site of the staged copy
    static __device__ const void *src(const Gauge32x12 &U, int blk, int lvb) { return U.p + ((size_t)blk * 12 << lvb); }
};
template <> struct F32Links<Gauge32x18> {
    static constexpr bool EXPAND = false;
    static constexpr int STAGE = 288;
    static __device__ const void *src(const Gauge32x18 &U, int blk, int lvb) { return U.p + ((size_t)blk * 36 << lvb); }
};

template <int LVB>
__host__ __device__ constexpr size_t f32_smem_bytes()
{
    return (size_t)(1 << LVB) * (288 + 96) + 96 * 4 + 16;
}

template <int MU, int SGN, int VB>
__device__ __forceinline__ void f32_hop(const float4 *rs, int n, const float2 *sL, int lk, Cx<float> acc[12])
{
    Cx<float> s[12], h[6], w[6], u[9];
#pragma unroll
    for (int k = 0; k < 6; ++k) {
        const float4 v = rs[k * VB + n];
        s[2 * k] = {v.x, v.y};
        s[2 * k + 1] = {v.z, v.w};
    }
    project<MU, SGN>(s, h);
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        const float2 v = sL[(MU * 9 + k) * VB + lk];
        u[k] = {v.x, v.y};
    }
    if (SGN < 0) su3_mul(u, h, w);
    else su3_dag_mul(u, h, w);
    reconstruct_add<MU, SGN>(acc, w);
}

template <int VB>
__device__ __forceinline__ void f32_hops(const float4 *rs, const float2 *sL, int l, const int nf[4], const int nb[4],
                                         Cx<float> acc[12])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = Cx<float>{0.f, 0.f};
    if (nf[0] >= 0) f32_hop<0, -1, VB>(rs, nf[0], sL, l, acc);
    if (nb[0] >= 0) f32_hop<0, +1, VB>(rs, nb[0], sL, nb[0], acc);
    if (nf[1] >= 0) f32_hop<1, -1, VB>(rs, nf[1], sL, l, acc);
    if (nb[1] >= 0) f32_hop<1, +1, VB>(rs, nb[1], sL, nb[1], acc);
    if (nf[2] >= 0) f32_hop<2, -1, VB>(rs, nf[2], sL, l, acc);
    if (nb[2] >= 0) f32_hop<2, +1, VB>(rs, nb[2], sL, nb[2], acc);
    if (nf[3] >= 0) f32_hop<3, -1, VB>(rs, nf[3], sL, l, acc);
    if (nb[3] >= 0) f32_hop<3, +1, VB>(rs, nb[3], sL, nb[3], acc);
}

// one domain solve of the FP32 kernel: domain jb of `colour`, right-hand side
// rr; C is the clover term (MR on D_B) or its inverse (Jacobi on A_B)
template <bool JAC, int LVB, class GA>
__device__ __forceinline__ void sap_f32_body(const Geom &g, const Spinor32 &b, const Spinor32 &x, const GA &U,
                                             const Clover32 &C, float kappa, int colour, int nmr, int x_zero,
                                             int *status, int jb, int rr)
{
    constexpr int VB = 1 << LVB;
    constexpr int LB = LVB / 4;
    using FL = F32Links<GA>;
    extern __shared__ __align__(128) unsigned char smem[];
    float2 *sL = reinterpret_cast<float2 *>(smem);           // [4][9][VB]
    float4 *rs = reinterpret_cast<float4 *>(sL + 36 * VB);   // [6][VB]
    float *red = reinterpret_cast<float *>(rs + 6 * VB);     // 96 floats
    uint64_t *bar = reinterpret_cast<uint64_t *>(red + 96);
    // the 12-real copy lands in the upper 192 B per site of the link area
    float4 *stage = reinterpret_cast<float4 *>(sL + 12 * VB);

    Geom gg = g;
    gg.lvb = LVB;
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LB;
    Spinor32 bb = shift_rhs(b, rr, g.V), xx = shift_rhs(x, rr, g.V);
    bb.lvb = LVB;
    xx.lvb = LVB;
    GA Ug = U;
    Ug.lvb = LVB;
    Clover32 Cg = C;
    Cg.lvb = LVB;
    int j = jb;
    const int half0 = g.NB[0] >> 1;
    int bc[4];
    const int m = j % half0;
    j /= half0;
    bc[1] = j % g.NB[1];
    j /= g.NB[1];
    bc[2] = j % g.NB[2];
    bc[3] = j / g.NB[2];
    bc[0] = 2 * m + ((colour + bc[1] + bc[2] + bc[3]) & 1);
    const int blk = block_index(gg, bc);
    const int l = threadIdx.x;
    const int i = (blk << LVB) | l;

    if (l == 0) mbar_init(bar, 1);
    __syncthreads();
    static_assert(FL::STAGE * VB % 16 == 0, "bulk copies move multiples of 16 bytes");
    if (l == 0) {
        const unsigned lbytes = FL::STAGE * VB;
        mbar_arrive_expect_tx(bar, lbytes);
        bulk_g2s(FL::EXPAND ? (void *)stage : (void *)sL, FL::src(U, blk, LVB), lbytes, bar);
    }
    // a programmatic dependent of the previous colour launch (as in the FP16
    // MR kernel): x is read only once that launch has completed
    asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    asm volatile("griddepcontrol.wait;" ::: "memory");

    int lc[4], cg[4];
    local_coords(gg, l, lc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) cg[mu] = (bc[mu] << LB) + lc[mu];

    // 1. hopping part of D x from global memory while the copy lands
    Cx<float> acc[12];
    if (!x_zero) hop_site<false>(gg, cg, i, xx, Ug, acc);

    const bool ok = mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
    if (!__syncthreads_and(ok)) {
        mbar_wait_bounded(bar, 0, WAIT_LIMIT_NS);
        if (l == 0) atomicOr(status, MGC_DEV_TIMEOUT);
        return;
    }
    if (FL::EXPAND) {
        // rows 0 and 1 of this site's four links, then row 2 = conj(row0 x row1)
        // written over the staged copy once every thread has read its own
        float4 st[12];
#pragma unroll
        for (int k = 0; k < 12; ++k) st[k] = stage[k * VB + l];
        __syncthreads();
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) {
            Cx<float> u[9];
#pragma unroll
            for (int k = 0; k < 3; ++k) {
                const float4 v = st[mu * 3 + k];
                u[2 * k] = {v.x, v.y};
                u[2 * k + 1] = {v.z, v.w};
            }
            reconstruct_row2(u);
#pragma unroll
            for (int k = 0; k < 9; ++k) sL[(mu * 9 + k) * VB + l] = make_float2(u[k].r, u[k].i);
        }
    }

    // r_B = b - D x on the domain (MR), or the residual of A = C^-1 D (Jacobi)
    Cx<float> rv[12];
    bb.load(i, rv);
    if (!x_zero) {
        Cx<float> xs[12], cx[12];
        xx.load(i, xs);
        if (JAC) {
            clover_site(Cg, i, acc, cx);  // C^-1 H x
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<float>{fmaf(kappa, cx[k].r, rv[k].r - xs[k].r), fmaf(kappa, cx[k].i, rv[k].i - xs[k].i)};
        } else {
            clover_site(Cg, i, xs, cx);
#pragma unroll
            for (int k = 0; k < 12; ++k)
                rv[k] = Cx<float>{rv[k].r - fmaf(-kappa, acc[k].r, cx[k].r),
                                  rv[k].i - fmaf(-kappa, acc[k].i, cx[k].i)};
        }
    }
    int nf[4], nb[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        int t[4] = {lc[0], lc[1], lc[2], lc[3]};
        t[mu] = lc[mu] + 1;
        nf[mu] = (t[mu] < (1 << LB)) ? local_index(gg, t) : -1;
        t[mu] = lc[mu] - 1;
        nb[mu] = (t[mu] >= 0) ? local_index(gg, t) : -1;
    }
#pragma unroll
    for (int k = 0; k < 6; ++k) rs[k * VB + l] = make_float4(rv[2 * k].r, rv[2 * k].i, rv[2 * k + 1].r, rv[2 * k + 1].i);
    Cx<float> e[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) e[k] = Cx<float>{0.f, 0.f};
    __syncthreads();

    // 2'. Jacobi on A_B with e in shared memory (rs): e_1 = r_B, then
    // e <- r_B + kappa C^-1 H_B e
    if (JAC) {
        if (nmr >= 1)
#pragma unroll
            for (int k = 0; k < 12; ++k) e[k] = rv[k];
        for (int it = 1; it < nmr; ++it) {
            f32_hops<VB>(rs, sL, l, nf, nb, acc);
            Cx<float> t[12];
            clover_site(Cg, i, acc, t);
            __syncthreads();  // every thread has read e before it is replaced
#pragma unroll
            for (int k = 0; k < 12; ++k) e[k] = Cx<float>{fmaf(kappa, t[k].r, rv[k].r), fmaf(kappa, t[k].i, rv[k].i)};
#pragma unroll
            for (int k = 0; k < 6; ++k)
                rs[k * VB + l] = make_float4(e[2 * k].r, e[2 * k].i, e[2 * k + 1].r, e[2 * k + 1].i);
            __syncthreads();
        }
        nmr = 0;
    }

    // 2. minimal residual on D_B
    for (int it = 0; it < nmr; ++it) {
        f32_hops<VB>(rs, sL, l, nf, nb, acc);
        Cx<float> rv2[12], p[12];
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            const float4 v = rs[k * VB + l];
            rv2[2 * k] = {v.x, v.y};
            rv2[2 * k + 1] = {v.z, v.w};
        }
        clover_site(Cg, i, rv2, p);
        // <p, r> and <p, p> in four partial sums each (shorter dependent chains)
        float sr[4] = {0.f, 0.f, 0.f, 0.f}, si[4] = {0.f, 0.f, 0.f, 0.f}, sq[4] = {0.f, 0.f, 0.f, 0.f};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            const int q = k & 3;
            p[k] = Cx<float>{fmaf(-kappa, acc[k].r, p[k].r), fmaf(-kappa, acc[k].i, p[k].i)};
            sr[q] = fmaf(p[k].r, rv2[k].r, fmaf(p[k].i, rv2[k].i, sr[q]));
            si[q] = fmaf(p[k].r, rv2[k].i, fmaf(-p[k].i, rv2[k].r, si[q]));
            sq[q] = fmaf(p[k].r, p[k].r, fmaf(p[k].i, p[k].i, sq[q]));
        }
        float pr = (sr[0] + sr[1]) + (sr[2] + sr[3]);
        float pi = (si[0] + si[1]) + (si[2] + si[3]);
        float pp = (sq[0] + sq[1]) + (sq[2] + sq[3]);
        if constexpr (VB >= 128) block_sum3_v4<VB>(pr, pi, pp, red);
        else block_sum3(pr, pi, pp, red);
        // a domain whose <p, p> is below FP32's normal range takes no step
        // (1 / <p, p> would overflow)
        const float ipp = pp >= FLT_MIN ? 1.0f / pp : 0.f;
        const Cx<float> alpha = {pr * ipp, pi * ipp};
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            e[k] = cfma(alpha, rv2[k], e[k]);
            rv2[k] = rv2[k] - alpha * p[k];
        }
#pragma unroll
        for (int k = 0; k < 6; ++k)
            rs[k * VB + l] = make_float4(rv2[2 * k].r, rv2[2 * k].i, rv2[2 * k + 1].r, rv2[2 * k + 1].i);
        __syncthreads();
    }

    // 3. x_B += e
    if (!x_zero) {
        Cx<float> xo[12];
        xx.load(i, xo);
#pragma unroll
        for (int k = 0; k < 12; ++k) e[k] = e[k] + xo[k];
    }
    xx.store(i, e);
}

template <bool JAC, int LVB, class GA>
__global__ void __launch_bounds__(1 << LVB, 2) k_sap_f32(Geom g, Spinor32 b, Spinor32 x, GA U, Clover32 C, float kappa,
                                                         int colour, int nmr, int x_zero, int *status)
{
    sap_f32_body<JAC, LVB>(g, b, x, U, C, kappa, colour, nmr, x_zero, status, blockIdx.x, blockIdx.y);
}

template <bool JAC, int LVB, class GA>
static int sap_run_f32(const mgc_clover_s *op, Spinor32 b, Spinor32 x, GA U, Clover32 C, int nrhs, int n_cy, int n_mr,
                       int x_is_zero, cudaStream_t s, int compress)
{
    const Geom &g = op->gauge->lat->g;
    constexpr size_t smem = f32_smem_bytes<LVB>();
    auto kern = k_sap_f32<JAC, LVB, GA>;
    MGC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(g.nblocks / 2, nrhs);
    // colour launches after the first are programmatic dependents of the one
    // before (griddepcontrol in the kernel)
    cudaLaunchAttribute pdl[1];
    pdl[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    pdl[0].val.programmaticStreamSerializationAllowed = 1;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = grid;
    cfg.blockDim = dim3(1 << LVB);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = s;
    cfg.attrs = pdl;
    cfg.numAttrs = 1;
    for (int cy = 0; cy < n_cy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int xz = (cy == 0 && colour == 0) ? x_is_zero : 0;
            if (cy > 0 || colour > 0)
                MGC_CUDA(cudaLaunchKernelEx(&cfg, kern, g, b, x, U, C, (float)op->kappa, colour, n_mr, xz,
                                            op->d_status));
            else
                kern<<<grid, 1 << LVB, smem, s>>>(g, b, x, U, C, (float)op->kappa, colour, n_mr, xz, op->d_status);
            count(1, sap_launch_bytes(g, 32, compress, nrhs, xz != 0));
        }
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

// FP16 storage: the compile-time kernel for cubic 2^4 and 4^4 domains
template <int MODE, class SP, class GA, class CL>
static int sap_run_staged(const mgc_clover_s *op, SP b, SP x, GA U, CL C, CL Ci, int nrhs, int n_cy, int n_mr,
                          int x_is_zero, cudaStream_t s, int prec, int compress);

template <bool JAC, class GA>
static int sap_dispatch16(const mgc_clover_s *op, Spinor16 b, Spinor16 x, GA U, Clover16 C, int nrhs, int n_cy,
                          int n_mr, int x_is_zero, cudaStream_t s, int compress)
{
    const Geom &g = op->gauge->lat->g;
    const bool cube = g.lb[0] == g.lb[1] && g.lb[1] == g.lb[2] && g.lb[2] == g.lb[3];
    if (cube && g.lvb == 8) return sap_run_h16<JAC, 8>(op, b, x, U, C, nrhs, n_cy, n_mr, x_is_zero, s, compress);
    if (cube && g.lvb == 4) return sap_run_h16<JAC, 4>(op, b, x, U, C, nrhs, n_cy, n_mr, x_is_zero, s, compress);
    return sap_run_staged<JAC ? SAP_JAC : SAP_MR>(op, b, x, U, C, C, nrhs, n_cy, n_mr, x_is_zero, s, 16, compress);
}

// ------------------------------------------------------------------ batches of lattices
// One launch covers one colour of every lattice of a batch and all their
// right-hand sides.  Thread block b belongs to the first lattice k with
// b < end[k]; within a lattice the order of (domain, right-hand side) pairs is
// chosen by the caller: rhs_fast = 1 puts the right-hand sides of one domain
// next to each other (they share the domain's links and clover term in L2).
template <class SP, class GA, class CL> struct SapBatch {
    int n;
    int rhs_fast;
    int end[MGC_BATCH_MAX];
    int nrhs[MGC_BATCH_MAX];
    int ndom[MGC_BATCH_MAX];  // domains of one colour
    Geom g[MGC_BATCH_MAX];
    SP b[MGC_BATCH_MAX], x[MGC_BATCH_MAX];
    GA U[MGC_BATCH_MAX];
    CL C[MGC_BATCH_MAX];
    float kappa[MGC_BATCH_MAX];
    int *status[MGC_BATCH_MAX];
};

template <class BT>
__device__ __forceinline__ void batch_item(const BT &B, int &k, int &jb, int &rr)
{
    k = 0;
    while (k < B.n - 1 && (int)blockIdx.x >= B.end[k]) ++k;
    const int local = blockIdx.x - (k ? B.end[k - 1] : 0);
    if (B.rhs_fast) {
        rr = local % B.nrhs[k];
        jb = local / B.nrhs[k];
    } else {
        jb = local % B.ndom[k];
        rr = local / B.ndom[k];
    }
}

template <int LVB, class GA>
__global__ void __launch_bounds__(1 << LVB, 2) k_sap_h16_batch(SapBatch<Spinor16, GA, Clover16> B, int colour, int nmr,
                                                               int x_zero)
{
    int k, jb, rr;
    batch_item(B, k, jb, rr);
    sap_m16_body<LVB>(B.g[k], B.b[k], B.x[k], B.U[k], B.C[k], B.kappa[k], colour, nmr, x_zero, B.status[k], jb, rr);
}

template <int LVB, class GA>
__global__ void __launch_bounds__(1 << LVB, 2) k_sap_f32_batch(SapBatch<Spinor32, GA, Clover32> B, int colour, int nmr,
                                                               int x_zero)
{
    int k, jb, rr;
    batch_item(B, k, jb, rr);
    sap_f32_body<false, LVB>(B.g[k], B.b[k], B.x[k], B.U[k], B.C[k], B.kappa[k], colour, nmr, x_zero, B.status[k], jb, rr);
}

// one block per SM: selecting the lattice at run time costs registers that a
// 128-register bound would turn into spills
template <class SP, class GA, class CL>
__global__ void __launch_bounds__(256, 1) k_sap_staged_batch(SapBatch<SP, GA, CL> B, int colour, int nmr, int x_zero)
{
    int k, jb, rr;
    batch_item(B, k, jb, rr);
    sap_staged_body<SAP_MR>(B.g[k], B.b[k], B.x[k], B.U[k], B.C[k], B.C[k], B.kappa[k], colour, nmr, x_zero, B.status[k], jb, rr);
}

template <class SP, class GA, class CL>
static void fill_batch(SapBatch<SP, GA, CL> &B, const BatchSpec &spec)
{
    B.n = spec.n;
    B.rhs_fast = spec.rhs_fast;
    int acc = 0;
    for (int k = 0; k < spec.n; ++k) {
        const mgc_clover_s *op = spec.ops[k];
        const Geom &g = op->gauge->lat->g;
        B.g[k] = g;
        B.nrhs[k] = spec.nrhs[k];
        B.ndom[k] = g.nblocks / 2;
        acc += B.ndom[k] * spec.nrhs[k];
        B.end[k] = acc;
        B.kappa[k] = (float)op->kappa;
        B.status[k] = op->d_status;
    }
}

static Spinor16 batch_sp16(const Geom &g, const void *p, int nrhs)
{
    uint4 *d = (uint4 *)p;
    return Spinor16{d, (float *)(d + (size_t)nrhs * g.V * 3), g.lvb};
}

int launch_sap_batch(const BatchSpec &spec, int prec, const void *const *b, void *const *x, int n_cy, int n_mr,
                     int x_is_zero, cudaStream_t s)
{
    const mgc_clover_s *op0 = spec.ops[0];
    const mgc_gauge_s *ga0 = op0->gauge;
    const Geom &g0 = ga0->lat->g;
    const int vb = 1 << g0.lvb;
    const bool cube = g0.lb[0] == g0.lb[1] && g0.lb[1] == g0.lb[2] && g0.lb[2] == g0.lb[3];
    int blocks = 0;
    double bytes_x0 = 0, bytes = 0;
    for (int k = 0; k < spec.n; ++k) {
        const Geom &g = spec.ops[k]->gauge->lat->g;
        blocks += g.nblocks / 2 * spec.nrhs[k];
        bytes_x0 += sap_launch_bytes(g, prec, ga0->compress, spec.nrhs[k], true);
        bytes += sap_launch_bytes(g, prec, ga0->compress, spec.nrhs[k], false);
    }
    auto run = [&](auto kern, auto &B, size_t smem) -> int {
        MGC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        for (int cy = 0; cy < n_cy; ++cy)
            for (int colour = 0; colour < 2; ++colour) {
                const int xz = (cy == 0 && colour == 0) ? x_is_zero : 0;
                kern<<<blocks, vb, smem, s>>>(B, colour, n_mr, xz);
                count(1, xz ? bytes_x0 : bytes);
            }
        MGC_CUDA(cudaGetLastError());
        return MGC_OK;
    };
    if (prec == 16) {
        if (ga0->compress == 12) {
            SapBatch<Spinor16, Gauge16x12, Clover16> B;
            fill_batch(B, spec);
            for (int k = 0; k < spec.n; ++k) {
                const mgc_clover_s *op = spec.ops[k];
                const Geom &g = op->gauge->lat->g;
                B.b[k] = batch_sp16(g, b[k], spec.nrhs[k]);
                B.x[k] = batch_sp16(g, x[k], spec.nrhs[k]);
                B.U[k] = Gauge16x12{(uint2 *)op->gauge->U16, g.lvb};
                B.C[k] = Clover16{(uint4 *)op->C16, op->C16_sc, g.lvb};
            }
            if (cube && g0.lvb == 8) return run(k_sap_h16_batch<8, Gauge16x12>, B, h16_smem_bytes<8>());
            if (cube && g0.lvb == 4) return run(k_sap_h16_batch<4, Gauge16x12>, B, h16_smem_bytes<4>());
            return run(k_sap_staged_batch<Spinor16, Gauge16x12, Clover16>, B, staged_smem<Gauge16x12, Clover16>(vb));
        }
        SapBatch<Spinor16, Gauge16x18, Clover16> B;
        fill_batch(B, spec);
        for (int k = 0; k < spec.n; ++k) {
            const mgc_clover_s *op = spec.ops[k];
            const Geom &g = op->gauge->lat->g;
            B.b[k] = batch_sp16(g, b[k], spec.nrhs[k]);
            B.x[k] = batch_sp16(g, x[k], spec.nrhs[k]);
            B.U[k] = Gauge16x18{(uint32_t *)op->gauge->U16, g.lvb};
            B.C[k] = Clover16{(uint4 *)op->C16, op->C16_sc, g.lvb};
        }
        if (cube && g0.lvb == 8) return run(k_sap_h16_batch<8, Gauge16x18>, B, h16_smem_bytes<8>());
        if (cube && g0.lvb == 4) return run(k_sap_h16_batch<4, Gauge16x18>, B, h16_smem_bytes<4>());
        return run(k_sap_staged_batch<Spinor16, Gauge16x18, Clover16>, B, staged_smem<Gauge16x18, Clover16>(vb));
    }
    if (prec != 32) return fail(MGC_ERR_INVALID_ARG, "batched smoother precision must be 32 or 16");
    if (ga0->compress == 12) {
        SapBatch<Spinor32, Gauge32x12, Clover32> B;
        fill_batch(B, spec);
        for (int k = 0; k < spec.n; ++k) {
            const mgc_clover_s *op = spec.ops[k];
            const Geom &g = op->gauge->lat->g;
            B.b[k] = Spinor32{(float4 *)b[k], g.lvb};
            B.x[k] = Spinor32{(float4 *)x[k], g.lvb};
            B.U[k] = Gauge32x12{(float4 *)op->gauge->U32, g.lvb};
            B.C[k] = Clover32{(float4 *)op->C32, g.lvb};
        }
        if (cube && g0.lvb == 8) return run(k_sap_f32_batch<8, Gauge32x12>, B, f32_smem_bytes<8>());
        if (cube && g0.lvb == 4) return run(k_sap_f32_batch<4, Gauge32x12>, B, f32_smem_bytes<4>());
        return run(k_sap_staged_batch<Spinor32, Gauge32x12, Clover32>, B, staged_smem<Gauge32x12, Clover32>(vb));
    }
    SapBatch<Spinor32, Gauge32x18, Clover32> B;
    fill_batch(B, spec);
    for (int k = 0; k < spec.n; ++k) {
        const mgc_clover_s *op = spec.ops[k];
        const Geom &g = op->gauge->lat->g;
        B.b[k] = Spinor32{(float4 *)b[k], g.lvb};
        B.x[k] = Spinor32{(float4 *)x[k], g.lvb};
        B.U[k] = Gauge32x18{(float2 *)op->gauge->U32, g.lvb};
        B.C[k] = Clover32{(float4 *)op->C32, g.lvb};
    }
    if (cube && g0.lvb == 8) return run(k_sap_f32_batch<8, Gauge32x18>, B, f32_smem_bytes<8>());
    if (cube && g0.lvb == 4) return run(k_sap_f32_batch<4, Gauge32x18>, B, f32_smem_bytes<4>());
    return run(k_sap_staged_batch<Spinor32, Gauge32x18, Clover32>, B, staged_smem<Gauge32x18, Clover32>(vb));
}

// Self-test of the bounded wait used above: one block waits on an mbarrier of
// arrival count 1; with arrive != 0 thread 0 arrives and the wait completes,
// with arrive == 0 nothing arrives and every thread gives up after limit_ns.
__global__ void k_wait_selftest(int arrive, unsigned long long limit_ns, int *status)
{
    __shared__ uint64_t bar;
    if (threadIdx.x == 0) mbar_init(&bar, 1);
    __syncthreads();
    if (arrive && threadIdx.x == 0) mbar_arrive(&bar);
    const bool ok = mbar_wait_bounded(&bar, 0, limit_ns);
    if (!__syncthreads_and(ok) && threadIdx.x == 0) atomicOr(status, MGC_DEV_TIMEOUT);
}

int selftest_bounded_wait(long long limit_ns, int arrive, int *flag_out, cudaStream_t s)
{
    int *d = nullptr;
    MGC_CUDA(cudaMalloc(&d, sizeof(int)));
    cudaMemsetAsync(d, 0, sizeof(int), s);
    k_wait_selftest<<<1, 64, 0, s>>>(arrive, (unsigned long long)limit_ns, d);
    cudaError_t e = cudaGetLastError();
    int h = 0;
    if (e == cudaSuccess) e = cudaMemcpyAsync(&h, d, sizeof(int), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    cudaFree(d);
    if (e != cudaSuccess) return cuda_fail(e, "bounded-wait self-test", __FILE__, __LINE__);
    count(1, 0.0);
    *flag_out = h;
    return h ? fail(MGC_ERR_TIMEOUT, "the self-test wait ran out as designed") : MGC_OK;
}

template <int MODE, class SP, class GA, class CL>
static int sap_run_staged(const mgc_clover_s *op, SP b, SP x, GA U, CL C, CL Ci, int nrhs, int n_cy, int n_mr,
                          int x_is_zero, cudaStream_t s, int prec, int compress)
{
    const Geom &g = op->gauge->lat->g;
    const int vb = 1 << g.lvb;
    const size_t smem = staged_smem<GA, CL>(vb);
    auto kern = k_sap_staged<MODE, SP, GA, CL>;
    MGC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(g.nblocks / 2, nrhs);
    for (int cy = 0; cy < n_cy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int xz = (cy == 0 && colour == 0) ? x_is_zero : 0;
            kern<<<grid, vb, smem, s>>>(g, b, x, U, C, Ci, (float)op->kappa, colour, n_mr, xz, op->d_status);
            count(1, sap_launch_bytes(g, prec, compress, nrhs, xz != 0));
        }
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

template <int MODE, class SP, class GA, class CL>
static int sap_run(const Geom &g, SP b, SP x, GA U, CL C, CL Ci, double kappa, int nrhs, int n_cy, int n_mr,
                   int x_is_zero,
                   cudaStream_t s, int prec, int compress)
{
    using T = typename SP::Real;
    const int vb = 1 << g.lvb;
    const size_t smem = (size_t)vb * 12 * sizeof(Cx<T>) + 96 * sizeof(T);
    auto kern = k_sap_colour<MODE, SP, GA, CL>;
    if (smem > 48 * 1024) MGC_CUDA(cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    dim3 grid(g.nblocks / 2, nrhs);
    for (int cy = 0; cy < n_cy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            const int xz = (cy == 0 && colour == 0) ? x_is_zero : 0;
            kern<<<grid, vb, smem, s>>>(g, b, x, U, C, Ci, (T)kappa, colour, n_mr, xz);
            count(1, sap_launch_bytes(g, prec, compress, nrhs, xz != 0));
        }
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

// the smoother: MR on D_B (clover C), Jacobi on A_B (clover C^-1) or even-odd
// MR on D_B (clover C, odd-site C^-1 from global memory)
template <int MODE>
static int sap_launch_impl(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_it,
                           int x_is_zero, cudaStream_t s)
{
    const mgc_gauge_s *ga = op->gauge;
    const Geom &g = ga->lat->g;
    constexpr bool jac = MODE == SAP_JAC;
    if ((1 << g.lvb) > 256) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "SAP domains are limited to 256 sites");
    if (prec == 64) {
        return sap_run<MODE>(g, Spinor64{(double2 *)b, g.lvb}, Spinor64{(double2 *)x, g.lvb}, Gauge64{ga->U64, g.lvb},
                             Clover64{jac ? op->Ci64 : op->C64, g.lvb}, Clover64{op->Ci64, g.lvb}, op->kappa, nrhs,
                             n_cy, n_it, x_is_zero, s, prec, ga->compress);
    }
    if (!has_prec(ga, prec)) return fail(MGC_ERR_INVALID_ARG, "no copy of the operator at this precision");
    // the FP32/FP16 kernels stage each domain's links and clover term with 1-D
    // bulk copies, which must start on 16-byte boundaries: the fields are
    // allocated that way and every domain's share is a multiple of 16 bytes
    const uintptr_t al = prec == 32 ? ((uintptr_t)ga->U32 | (uintptr_t)op->C32 | (uintptr_t)op->Ci32)
                                    : ((uintptr_t)ga->U16 | (uintptr_t)op->C16 | (uintptr_t)op->C16_sc |
                                       (uintptr_t)op->Ci16 | (uintptr_t)op->Ci16_sc);
    if ((al & 15) || (1 << g.lvb) % 4)
        return fail(MGC_ERR_INVALID_ARG, "smoother fields not aligned for bulk copies");
    const int cp = ga->compress;
    if (prec == 32) {
        Spinor32 B{(float4 *)b, g.lvb}, X{(float4 *)x, g.lvb};
        Clover32 C{(float4 *)(jac ? op->Ci32 : op->C32), g.lvb}, Ci{(float4 *)op->Ci32, g.lvb};
        const bool cube = g.lb[0] == g.lb[1] && g.lb[1] == g.lb[2] && g.lb[2] == g.lb[3];
        if (MODE != SAP_EO && cube && (g.lvb == 8 || g.lvb == 4)) {
            const Gauge32x12 U12{(float4 *)ga->U32, g.lvb};
            const Gauge32x18 U18{(float2 *)ga->U32, g.lvb};
            if (g.lvb == 8)
                return cp == 12 ? sap_run_f32<jac, 8>(op, B, X, U12, C, nrhs, n_cy, n_it, x_is_zero, s, cp)
                                : sap_run_f32<jac, 8>(op, B, X, U18, C, nrhs, n_cy, n_it, x_is_zero, s, cp);
            return cp == 12 ? sap_run_f32<jac, 4>(op, B, X, U12, C, nrhs, n_cy, n_it, x_is_zero, s, cp)
                            : sap_run_f32<jac, 4>(op, B, X, U18, C, nrhs, n_cy, n_it, x_is_zero, s, cp);
        }
        if (cp == 12)
            return sap_run_staged<MODE>(op, B, X, Gauge32x12{(float4 *)ga->U32, g.lvb}, C, Ci, nrhs, n_cy, n_it,
                                        x_is_zero, s, prec, cp);
        return sap_run_staged<MODE>(op, B, X, Gauge32x18{(float2 *)ga->U32, g.lvb}, C, Ci, nrhs, n_cy, n_it,
                                    x_is_zero, s, prec, cp);
    }
    const size_t nV = (size_t)nrhs * g.V;
    Spinor16 B{(uint4 *)b, (float *)((uint4 *)b + nV * 3), g.lvb};
    Spinor16 X{(uint4 *)x, (float *)((uint4 *)x + nV * 3), g.lvb};
    const Clover16 Ci{(uint4 *)op->Ci16, op->Ci16_sc, g.lvb};
    const Clover16 C = jac ? Ci : Clover16{(uint4 *)op->C16, op->C16_sc, g.lvb};
    if (MODE == SAP_EO) {
        if (cp == 12)
            return sap_run_staged<SAP_EO>(op, B, X, Gauge16x12{(uint2 *)ga->U16, g.lvb}, C, Ci, nrhs, n_cy, n_it,
                                          x_is_zero, s, 16, cp);
        return sap_run_staged<SAP_EO>(op, B, X, Gauge16x18{(uint32_t *)ga->U16, g.lvb}, C, Ci, nrhs, n_cy, n_it,
                                      x_is_zero, s, 16, cp);
    }
    if (cp == 12)
        return sap_dispatch16<jac>(op, B, X, Gauge16x12{(uint2 *)ga->U16, g.lvb}, C, nrhs, n_cy, n_it, x_is_zero, s,
                                   cp);
    return sap_dispatch16<jac>(op, B, X, Gauge16x18{(uint32_t *)ga->U16, g.lvb}, C, nrhs, n_cy, n_it, x_is_zero, s,
                               cp);
}

int launch_sap(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_mr, int x_is_zero,
               cudaStream_t s)
{
    return sap_launch_impl<SAP_MR>(op, prec, b, x, nrhs, n_cy, n_mr, x_is_zero, s);
}

int launch_sap_A(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_jacobi,
                 int x_is_zero, cudaStream_t s)
{
    return sap_launch_impl<SAP_JAC>(op, prec, b, x, nrhs, n_cy, n_jacobi, x_is_zero, s);
}

int launch_sap_eo(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_mr,
                  int x_is_zero, cudaStream_t s)
{
    return sap_launch_impl<SAP_EO>(op, prec, b, x, nrhs, n_cy, n_mr, x_is_zero, s);
}

}  // namespace mgc
