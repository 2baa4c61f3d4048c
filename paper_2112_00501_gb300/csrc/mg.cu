// Two-level multigrid (Sec. 3) in FP32 arithmetic: null-vector basis,
// restriction and prolongation, the Galerkin coarse operator as a 9-point
// stencil, a coarse BiCGStab, the two-level preconditioner (coarse correction,
// then QWS's SAP for A as post-smoother) and its setup.
//
// Fine fields are FP32 packed spinors (block-major, 6 float4 planes per
// domain); chirality 0 (spins 0, 1) is planes 0..2, chirality 1 planes 3..5.
// Aggregates are unions of whole SAP domains, so one thread block of one
// thread per domain site walks an aggregate's domains.  Coarse vectors are
// float2 [Vc][2][nvec]; the coarse stencil is float2 [Vc][9][column][row]
// (column-major blocks, so the threads of a coarse matrix-vector product read
// consecutive rows).  Reductions of coarse vectors run in FP64 with a fixed
// grid and a fixed-order second pass.
#include <cmath>
#include <type_traits>
#include <vector>

#include "hop.cuh"
#include "mgc_host.h"

namespace mgc {
namespace {

constexpr int CHUNK = 8;    // null vectors per restriction pass
constexpr int RWARPS = 8;   // aggregates (one warp each) per restriction block
constexpr int CRT = 256;    // threads of the coarse reductions
constexpr int CRG = 64;     // blocks of the coarse reductions


struct MgGeom {
    Geom g;          // fine lattice
    int ratio[4];    // SAP domains per aggregate per direction
    int Lc[4];       // coarse lattice
    int Vc, nvec, n2, da;  // coarse sites, vectors, 2 nvec, domains per aggregate
};

// masked FP32 spinor: only the components of one chirality
struct Chiral32 {
    Spinor32 b;
    int chi;
    using Real = float;
    __device__ __forceinline__ void load(int i, Cx<float> s[12]) const
    {
        b.load(i, s);
#pragma unroll
        for (int k = 0; k < 12; ++k)
            if ((k / 6) != chi) s[k] = Cx<float>{0.f, 0.f};
    }
};

__device__ __forceinline__ int coarse_index(const MgGeom &m, const int a[4])
{
    return a[0] + m.Lc[0] * (a[1] + m.Lc[1] * (a[2] + m.Lc[2] * a[3]));
}

// the d-th SAP domain of aggregate ac (coarse coordinates)
__device__ __forceinline__ int agg_domain(const MgGeom &m, const int ac[4], int d)
{
    int bc[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        bc[mu] = ac[mu] * m.ratio[mu] + d % m.ratio[mu];
        d /= m.ratio[mu];
    }
    return block_index(m.g, bc);
}

__device__ __forceinline__ void coarse_coords(const MgGeom &m, int a, int ac[4])
{
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        ac[mu] = a % m.Lc[mu];
        a /= m.Lc[mu];
    }
}

// whether fine site c lies on the face of its aggregate that coarse stencil
// entry k >= 1 crosses (the +mu face for k = 1 + 2 mu, the -mu face for
// k = 2 + 2 mu): the only sites where that entry's field is nonzero
__device__ __forceinline__ bool on_face(const MgGeom &m, const int c[4], int k)
{
    const int mu = (k - 1) / 2;
    const int A = m.ratio[mu] << m.g.lb[mu];  // aggregate extent along mu
    return ((k - 1) % 2 == 0) ? ((c[mu] + 1) % A == 0) : (c[mu] % A == 0);
}

__device__ __forceinline__ int aggregate_of(const MgGeom &m, int i)
{
    int bc[4], ac[4];
    block_coords(m.g, i >> m.g.lvb, bc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) ac[mu] = bc[mu] / m.ratio[mu];
    return coarse_index(m, ac);
}

__device__ __forceinline__ const float4 *plane(const float4 *f, const Geom &g, int i, int k)
{
    return f + ((size_t)(i >> g.lvb) * 6 + k << g.lvb) + (i & ((1 << g.lvb) - 1));
}

// sum over the lanes of a warp; a block smaller than a warp (16 threads for
// 2^4 domains) reduces over its own lanes only
__device__ __forceinline__ float warp_sum(float v)
{
    const int n = blockDim.x < 32 ? blockDim.x : 32;
    const unsigned mask = n == 32 ? 0xffffffffu : ((1u << n) - 1u);
    for (int o = n >> 1; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, n);
    return v;
}

// conj(a) b for the two complex numbers of a float4, accumulated
__device__ __forceinline__ void cdot4(float &re, float &im, float4 a, float4 b)
{
    re = fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, fmaf(a.w, b.w, re))));
    im = fmaf(a.x, b.y, fmaf(-a.y, b.x, fmaf(a.z, b.w, fmaf(-a.w, b.z, im))));
}

// ------------------------------------------------------------------ restriction
// out[a][chi][j] = sum_{x in a} conj(W_j(x))_chi . v(x)_chi for the vectors
// j0 .. j0 + CHUNK - 1; one warp per (aggregate, chunk), RWARPS aggregates per
// thread block.  With colq >= 0 the result goes to column colq of the coarse
// stencil entry k instead (Dc[a][k][colq][row]), and for k >= 1 only the face
// sites where that entry's field lives are read.
template <int NCOL>
__global__ void __launch_bounds__(RWARPS * 32) k_restrict(MgGeom m, const float4 *W, const float4 *v, const float4 *v2,
                                                          float2 *out, float2 *Dc, int k, int colq)
{
    // NCOL = 2: two coarse-operator columns (fields v and v2, columns colq and
    // colq + 1 of entry k) share each read of the basis
    // one warp per aggregate: each lane takes every 32nd site of it and keeps
    // the 2 x CHUNK complex sums, reduced across the warp once at the end
    const int lane = threadIdx.x & 31;
    const int a = blockIdx.x * RWARPS + (threadIdx.x >> 5);
    if (a >= m.Vc) return;
    const int j0 = blockIdx.y * CHUNK;
    const size_t fs = (size_t)m.g.V * 6;  // float4 per field
    const int vb = 1 << m.g.lvb;
    int ac[4];
    coarse_coords(m, a, ac);
    float acc[NCOL][2][CHUNK][2];
#pragma unroll
    for (int f = 0; f < NCOL; ++f)
#pragma unroll
        for (int c = 0; c < 2; ++c)
#pragma unroll
            for (int j = 0; j < CHUNK; ++j) acc[f][c][j][0] = acc[f][c][j][1] = 0.f;
    // the sums of one site
    auto site = [&](int i) {
        float4 vv[NCOL][6];
#pragma unroll
        for (int q = 0; q < 6; ++q) {
            vv[0][q] = __ldg(plane(v, m.g, i, q));
            if (NCOL == 2) vv[NCOL - 1][q] = __ldg(plane(v2, m.g, i, q));
        }
#pragma unroll
        for (int j = 0; j < CHUNK; ++j) {
            if (j0 + j >= m.nvec) break;
            const float4 *w = W + (j0 + j) * fs;
#pragma unroll
            for (int q = 0; q < 6; ++q) {
                const float4 wq = __ldg(plane(w, m.g, i, q));
#pragma unroll
                for (int f = 0; f < NCOL; ++f) cdot4(acc[f][q / 3][j][0], acc[f][q / 3][j][1], wq, vv[f][q]);
            }
        }
    };
    if (colq >= 0 && k >= 1) {
        // a coarse-operator column's face field: it lives on the aggregate's
        // last (forward hop) or first (backward hop) layer along mu, i.e. on
        // one layer of the domains at that end; the lanes walk that layer only
        const int mu = (k - 1) / 2;
        const bool fwd = (k - 1) % 2 == 0;
        const int dmu = fwd ? m.ratio[mu] - 1 : 0;
        const int lmu = fwd ? (1 << m.g.lb[mu]) - 1 : 0;
        const int nface = vb >> m.g.lb[mu];
        for (int d = 0; d < m.da; ++d) {
            int rest = d, dc = 0;
#pragma unroll
            for (int nu = 0; nu < 4; ++nu) {
                if (nu == mu) dc = rest % m.ratio[nu];
                rest /= m.ratio[nu];
            }
            if (dc != dmu) continue;
            const int base = agg_domain(m, ac, d) << m.g.lvb;
            for (int t = lane; t < nface; t += 32) {
                int lc[4], r = t;
#pragma unroll
                for (int nu = 0; nu < 4; ++nu) {
                    if (nu == mu) {
                        lc[nu] = lmu;
                    } else {
                        lc[nu] = r & ((1 << m.g.lb[nu]) - 1);
                        r >>= m.g.lb[nu];
                    }
                }
                site(base | local_index(m.g, lc));
            }
        }
    } else {
        for (int d = 0; d < m.da; ++d) {
            const int base = agg_domain(m, ac, d) << m.g.lvb;
            for (int l = lane; l < vb; l += 32) site(base | l);
        }
    }
    // butterfly sums leave every total in every lane; lane t stores sum t of
    // each column
    constexpr int NVAL = 2 * CHUNK * 2;
    static_assert(NVAL == 32, "one sum per lane");
    const int chi = lane / (2 * CHUNK), j = (lane / 2) % CHUNK, ri = lane & 1;
#pragma unroll
    for (int f = 0; f < NCOL; ++f) {
        float *flat = &acc[f][0][0][0];
        float mine = 0.f;
#pragma unroll
        for (int t = 0; t < NVAL; ++t) {
            float x = flat[t];
#pragma unroll
            for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
            if (t == lane) mine = x;
        }
        if (j0 + j < m.nvec) {
            const int row = chi * m.nvec + j0 + j;
            float *dst = colq < 0
                             ? reinterpret_cast<float *>(out + (size_t)a * m.n2 + row)
                             : reinterpret_cast<float *>(Dc + (((size_t)a * 9 + k) * m.n2 + colq + f) * m.n2 + row);
            dst[ri] = mine;
        }
    }
}

// ------------------------------------------------------------------ prolongation
// v(x) = sum_j W_j(x)_chi u[a(x)][chi][j] (add != 0: v += P u)
__global__ void k_prolong(MgGeom m, const float4 *W, const float2 *u, float4 *v, int add)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.g.V) return;
    const int a = aggregate_of(m, i);
    const size_t fs = (size_t)m.g.V * 6;
    const float2 *ua = u + (size_t)a * m.n2;
#pragma unroll
    for (int q = 0; q < 6; ++q) {
        const int chi = q / 3;
        float4 acc = add ? *plane(v, m.g, i, q) : make_float4(0.f, 0.f, 0.f, 0.f);
        for (int j = 0; j < m.nvec; ++j) {
            const float2 c = __ldg(ua + chi * m.nvec + j);
            const float4 w = __ldg(plane(W + j * fs, m.g, i, q));
            acc.x = fmaf(w.x, c.x, fmaf(-w.y, c.y, acc.x));
            acc.y = fmaf(w.x, c.y, fmaf(w.y, c.x, acc.y));
            acc.z = fmaf(w.z, c.x, fmaf(-w.w, c.y, acc.z));
            acc.w = fmaf(w.z, c.y, fmaf(w.w, c.x, acc.w));
        }
        *const_cast<float4 *>(plane(v, m.g, i, q)) = acc;
    }
}

// ------------------------------------------------------------------ block Gram-Schmidt
// For every (aggregate, chirality), W_i -= <W_j, W_i> W_j (j < i), then W_i /= |W_i|,
// restricted to the aggregate and chirality; one thread block per
// (aggregate, chirality), one thread per domain site.  *bad counts the
// restrictions left with less than 1e-5 of their norm after the projections
// (linearly dependent to FP32 accuracy).
__device__ __forceinline__ float2 block_sum2(float a, float b, float *red)
{
    a = warp_sum(a);
    b = warp_sum(b);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, nw = (blockDim.x + 31) >> 5;
    __syncthreads();
    if (lane == 0) {
        red[2 * warp] = a;
        red[2 * warp + 1] = b;
    }
    __syncthreads();
    float sa = 0.f, sb = 0.f;
    for (int w = 0; w < nw; ++w) {
        sa += red[2 * w];
        sb += red[2 * w + 1];
    }
    return make_float2(sa, sb);
}

__global__ void k_block_gs(MgGeom m, float4 *W, int *bad)
{
    __shared__ float red[64];
    const int a = blockIdx.x, chi = blockIdx.y, l = threadIdx.x;
    const size_t fs = (size_t)m.g.V * 6;
    int ac[4];
    coarse_coords(m, a, ac);
    auto norm2 = [&](const float4 *wi) {
        float n2 = 0.f, dummy = 0.f;
        for (int d = 0; d < m.da; ++d) {
            const int s = (agg_domain(m, ac, d) << m.g.lvb) | l;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                const float4 t = *plane(wi, m.g, s, 3 * chi + q);
                n2 = fmaf(t.x, t.x, fmaf(t.y, t.y, fmaf(t.z, t.z, fmaf(t.w, t.w, n2))));
            }
        }
        return block_sum2(n2, dummy, red).x;
    };
    for (int i = 0; i < m.nvec; ++i) {
        float4 *wi = W + i * fs;
        const float n0 = norm2(wi);
        for (int j = 0; j < i; ++j) {
            const float4 *wj = W + j * fs;
            float re = 0.f, im = 0.f;
            for (int d = 0; d < m.da; ++d) {
                const int s = (agg_domain(m, ac, d) << m.g.lvb) | l;
#pragma unroll
                for (int q = 0; q < 3; ++q)
                    cdot4(re, im, *plane(wj, m.g, s, 3 * chi + q), *plane(wi, m.g, s, 3 * chi + q));
            }
            const float2 dd = block_sum2(re, im, red);
            for (int d = 0; d < m.da; ++d) {
                const int s = (agg_domain(m, ac, d) << m.g.lvb) | l;
#pragma unroll
                for (int q = 0; q < 3; ++q) {
                    float4 *p = const_cast<float4 *>(plane(wi, m.g, s, 3 * chi + q));
                    const float4 u = *plane(wj, m.g, s, 3 * chi + q);
                    float4 t = *p;
                    t.x -= dd.x * u.x - dd.y * u.y;
                    t.y -= dd.x * u.y + dd.y * u.x;
                    t.z -= dd.x * u.z - dd.y * u.w;
                    t.w -= dd.x * u.w + dd.y * u.z;
                    *p = t;
                }
            }
        }
        const float nn = norm2(wi);
        if (!(nn > 1e-10f * n0)) {
            if (l == 0) atomicAdd(bad, 1);
            continue;
        }
        const float inv = rsqrtf(nn);
        for (int d = 0; d < m.da; ++d) {
            const int s = (agg_domain(m, ac, d) << m.g.lvb) | l;
#pragma unroll
            for (int q = 0; q < 3; ++q) {
                float4 *p = const_cast<float4 *>(plane(wi, m.g, s, 3 * chi + q));
                float4 t = *p;
                t.x *= inv;
                t.y *= inv;
                t.z *= inv;
                t.w *= inv;
                *p = t;
            }
        }
    }
}

// ------------------------------------------------------------------ coarse operator columns
// H = the part of D that stencil entry k collects, applied at every fine site
// to p = W_i restricted to chirality chi: k = 0 the clover term and the hops
// that stay inside the aggregate, k = 1 + 2 mu the hop from x + mu across the
// aggregate's +mu face, k = 2 + 2 mu the hop from x - mu across its -mu face.
template <class GA>
__global__ void k_stencil_field(MgGeom m, Chiral32 p, GA U, Clover32 C, float kappa, int k, float4 *H)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= m.g.V) return;
    const Geom &g = m.g;
    int c[4];
    site_coords(g, i, c);
    // entries k >= 1 are zero off their face; the restriction of the column
    // reads face sites only, so nothing is stored elsewhere
    if (k >= 1 && !on_face(m, c, k)) return;
    Cx<float> acc[12];
#pragma unroll
    for (int q = 0; q < 12; ++q) acc[q] = Cx<float>{0.f, 0.f};
    // hops: acc += (1 -/+ gamma) U psi; selected per direction below
    auto hop = [&](auto MUc, int dir) {
        constexpr int MU = decltype(MUc)::value;
        bool wr;
        Cx<float> h[6], w[6], u[9];
        const int j = neighbour(g, c, MU, dir, &wr);
        const bool flip = MU == 3 && wr && g.tbc < 0;
        if (dir > 0) {
            load_project<MU, -1>(p, j, flip, h);
            U.load(i, MU, u);
            su3_mul(u, h, w);
            reconstruct_add<MU, -1>(acc, w);
        } else {
            load_project<MU, +1>(p, j, flip, h);
            U.load(j, MU, u);
            su3_dag_mul(u, h, w);
            reconstruct_add<MU, +1>(acc, w);
        }
    };
    auto inside = [&](int mu, int dir) {
        const int A = m.ratio[mu] << g.lb[mu];  // aggregate extent
        return dir > 0 ? ((c[mu] + 1) % A != 0) : (c[mu] % A != 0);
    };
    auto do_dir = [&](int mu, int dir) {
        if (mu == 0) hop(std::integral_constant<int, 0>{}, dir);
        else if (mu == 1) hop(std::integral_constant<int, 1>{}, dir);
        else if (mu == 2) hop(std::integral_constant<int, 2>{}, dir);
        else hop(std::integral_constant<int, 3>{}, dir);
    };
    Cx<float> out[12];
    if (k == 0) {
        for (int mu = 0; mu < 4; ++mu)
            for (int dir = -1; dir <= 1; dir += 2)
                if (inside(mu, dir)) do_dir(mu, dir);
        Cx<float> psi[12];
        p.load(i, psi);
        clover_site(C, i, psi, out);
#pragma unroll
        for (int q = 0; q < 12; ++q)
            out[q] = Cx<float>{fmaf(-kappa, acc[q].r, out[q].r), fmaf(-kappa, acc[q].i, out[q].i)};
    } else {
        const int mu = (k - 1) / 2, dir = ((k - 1) % 2 == 0) ? +1 : -1;
        if (!inside(mu, dir)) do_dir(mu, dir);
#pragma unroll
        for (int q = 0; q < 12; ++q) out[q] = Cx<float>{-kappa * acc[q].r, -kappa * acc[q].i};
    }
    Spinor32{H, g.lvb}.store(i, out);
}

// ------------------------------------------------------------------ coarse matrix-vector product
// out[a][r] = sum_k sum_q Dc[a][k][q][r] u[nbr_k(a)][q]; one thread per row,
// one thread block of n2 threads per coarse site
__global__ void k_coarse_apply(MgGeom m, const float2 *Dc, const float2 *u, float2 *out)
{
    const int a = blockIdx.x, r = threadIdx.x;
    if (r >= m.n2) return;
    int ac[4];
    coarse_coords(m, a, ac);
    float re = 0.f, im = 0.f;
    for (int k = 0; k < 9; ++k) {
        int nc[4] = {ac[0], ac[1], ac[2], ac[3]};
        if (k > 0) {
            const int mu = (k - 1) / 2, dir = ((k - 1) % 2 == 0) ? +1 : -1;
            nc[mu] = (nc[mu] + dir + m.Lc[mu]) % m.Lc[mu];
        }
        const float2 *ub = u + (size_t)coarse_index(m, nc) * m.n2;
        const float2 *col = Dc + ((size_t)a * 9 + k) * m.n2 * m.n2 + r;
        for (int q = 0; q < m.n2; ++q) {
            const float2 d = __ldg(col + (size_t)q * m.n2), x = __ldg(ub + q);
            re = fmaf(d.x, x.x, fmaf(-d.y, x.y, re));
            im = fmaf(d.x, x.y, fmaf(d.y, x.x, im));
        }
    }
    out[(size_t)a * m.n2 + r] = make_float2(re, im);
}

// ------------------------------------------------------------------ coarse vector reductions
template <int NV, class F>
__global__ void __launch_bounds__(CRT) k_creduce(int n, F f, double *partial)
{
    static_assert(NV <= 4, "the coarse partial-sum area holds four accumulators per block");
    __shared__ double sh[NV][CRT / 32];
    double acc[NV];
#pragma unroll
    for (int t = 0; t < NV; ++t) acc[t] = 0;
    for (int e = blockIdx.x * CRT + threadIdx.x; e < n; e += gridDim.x * CRT) f(e, acc);
#pragma unroll
    for (int t = 0; t < NV; ++t)
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], o);
    const int w = threadIdx.x >> 5;
    if ((threadIdx.x & 31) == 0)
#pragma unroll
        for (int t = 0; t < NV; ++t) sh[t][w] = acc[t];
    __syncthreads();
    if (threadIdx.x == 0)
#pragma unroll
        for (int t = 0; t < NV; ++t) {
            double s = 0;
            for (int q = 0; q < CRT / 32; ++q) s += sh[t][q];
            partial[blockIdx.x * NV + t] = s;
        }
}

// device-side BiCGStab scalars of the coarse solve (FP64):
// rho, <r0, v>, ||t||^2, <t, s>, ||r||^2, <r0, r_new>
enum { CS_RHO = 0, CS_R0V = 2, CS_TT = 4, CS_TS = 5, CS_RR = 7, CS_RHO1 = 8, CS_N = 10 };
__device__ __forceinline__ double2 ldz(const double *p) { return make_double2(p[0], p[1]); }
__device__ __forceinline__ double2 zdiv(double2 a, double2 b)
{
    const double n = b.x * b.x + b.y * b.y;
    return n > 0 ? make_double2((a.x * b.x + a.y * b.y) / n, (a.y * b.x - a.x * b.y) / n) : make_double2(0, 0);
}
__device__ __forceinline__ double2 zmul(double2 a, double2 b)
{
    return make_double2(a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x);
}
__device__ __forceinline__ float2 tof(double2 a) { return make_float2((float)a.x, (float)a.y); }
// alpha = rho / <r0, v>; omega = <t, s> / ||t||^2
__device__ __forceinline__ double2 cs_alpha(const double *sc) { return zdiv(ldz(sc + CS_RHO), ldz(sc + CS_R0V)); }
__device__ __forceinline__ double2 cs_omega(const double *sc)
{
    return sc[CS_TT] > 0 ? make_double2(sc[CS_TS] / sc[CS_TT], sc[CS_TS + 1] / sc[CS_TT]) : make_double2(0, 0);
}

template <int NV>
__global__ void k_cfinish(const double *partial, double *out, int nblk = CRG)
{
    if (threadIdx.x >= NV) return;
    double s = 0;
    for (int b = 0; b < nblk; ++b) s += partial[b * NV + threadIdx.x];
    out[threadIdx.x] = s;
}

template <class F>
__global__ void k_cmap(int n, F f)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x) f(e);
}

__device__ __forceinline__ void ddot(double *acc, float2 a, float2 b)
{
    acc[0] += (double)a.x * b.x + (double)a.y * b.y;
    acc[1] += (double)a.x * b.y - (double)a.y * b.x;
}
__device__ __forceinline__ float2 cmad(float2 c, float2 x, float2 y)  // y + c x
{
    return make_float2(fmaf(c.x, x.x, fmaf(-c.y, x.y, y.x)), fmaf(c.x, x.y, fmaf(c.y, x.x, y.y)));
}

// FP32 fine-field maps: v = a - b, v += b
__global__ void k_fsub(long long n4, const float4 *a, const float4 *b, float4 *v)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n4; e += (long long)gridDim.x * blockDim.x) {
        const float4 x = a[e], y = b[e];
        v[e] = make_float4(x.x - y.x, x.y - y.y, x.z - y.z, x.w - y.w);
    }
}
__global__ void k_fadd(long long n4, const float4 *b, float4 *v)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n4; e += (long long)gridDim.x * blockDim.x) {
        const float4 x = v[e], y = b[e];
        v[e] = make_float4(x.x + y.x, x.y + y.y, x.z + y.z, x.w + y.w);
    }
}
__global__ void k_fscale(long long n4, float s, float4 *v)
{
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < n4; e += (long long)gridDim.x * blockDim.x) {
        const float4 x = v[e];
        v[e] = make_float4(s * x.x, s * x.y, s * x.z, s * x.w);
    }
}
// ||v||^2 of a fine FP32 field: FNG blocks (every SM busy, within the
// partial area of CRG * 4 doubles), FP32 partial sums over four float4 per
// step, FP64 beyond
constexpr int FNG = CRG * 4;
__global__ void __launch_bounds__(CRT) k_fnorm2(long long n4, const float4 *v, double *partial)
{
    __shared__ double sh[CRT / 32];
    double acc = 0;
    const long long stride = (long long)gridDim.x * CRT;
    long long e = blockIdx.x * (long long)CRT + threadIdx.x;
    for (; e + 3 * stride < n4; e += 4 * stride) {
        float f = 0.f;
#pragma unroll
        for (int u = 0; u < 4; ++u) {
            const float4 x = v[e + u * stride];
            f = fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, fmaf(x.w, x.w, f))));
        }
        acc += (double)f;
    }
    for (; e < n4; e += stride) {
        const float4 x = v[e];
        acc += (double)fmaf(x.x, x.x, fmaf(x.y, x.y, fmaf(x.z, x.z, x.w * x.w)));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(0xffffffffu, acc, o);
    if ((threadIdx.x & 31) == 0) sh[threadIdx.x >> 5] = acc;
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0;
        for (int q = 0; q < CRT / 32; ++q) s += sh[q];
        partial[blockIdx.x] = s;
    }
}

// canonical complex128 <-> FP32 coarse vectors and the stencil export
__global__ void k_c64_to32(int n, const double2 *in, float2 *out)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        out[e] = make_float2((float)in[e].x, (float)in[e].y);
}
__global__ void k_c32_to64(int n, const float2 *in, double2 *out)
{
    for (int e = blockIdx.x * blockDim.x + threadIdx.x; e < n; e += gridDim.x * blockDim.x)
        out[e] = make_double2(in[e].x, in[e].y);
}
__global__ void k_export_stencil(int nblk, int n2, const float2 *Dc, double2 *out)
{
    const long long tot = (long long)nblk * n2 * n2;
    for (long long e = blockIdx.x * (long long)blockDim.x + threadIdx.x; e < tot; e += (long long)gridDim.x * blockDim.x) {
        const long long b = e / ((long long)n2 * n2);
        const int rem = (int)(e % ((long long)n2 * n2)), row = rem / n2, col = rem % n2;
        const float2 v = Dc[(b * n2 + col) * n2 + row];
        out[e] = make_double2(v.x, v.y);
    }
}

inline int fgrid(long long n, int t) { long long g = (n + t - 1) / t; return (int)(g < 4096 ? (g < 1 ? 1 : g) : 4096); }

}  // namespace

// ------------------------------------------------------------------ handle
struct MgWork {
    float4 *W = nullptr, *Vraw = nullptr;
    float2 *Dc = nullptr;
    float2 *cb = nullptr, *cx = nullptr, *cr = nullptr, *cr0 = nullptr, *cp = nullptr, *cv = nullptr,
           *cs = nullptr, *ct = nullptr;
    float4 *f0 = nullptr, *f1 = nullptr, *f2 = nullptr, *f3 = nullptr, *f4 = nullptr;
    void *l16a = nullptr, *l16b = nullptr;  // FP16 smoother fields
    double2 *d0 = nullptr, *d1 = nullptr;   // FP64 fine work
    double *partial = nullptr, *scal = nullptr, *hscal = nullptr;
    int *dbad = nullptr;
};

}  // namespace mgc

using namespace mgc;

struct mgc_mg_s {
    mgc_clover_s *op;
    MgGeom m;
    MgWork w;
    int ready = 0;
};

namespace mgc {
namespace {

size_t fine32_bytes(const mgc_mg_s *M) { return (size_t)M->m.g.V * 96; }
long long fine4(const mgc_mg_s *M) { return (long long)M->m.g.V * 6; }
int ncoarse(const mgc_mg_s *M) { return M->m.Vc * M->m.n2; }

int read_scalars(mgc_mg_s *M, int nd, double *out, cudaStream_t s)
{
    MGC_CUDA(cudaMemcpyAsync(M->w.hscal, M->w.scal, nd * sizeof(double), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    for (int k = 0; k < nd; ++k) out[k] = M->w.hscal[k];
    return MGC_OK;
}

template <int NV, class F>
int creduce(mgc_mg_s *M, F f, cudaStream_t s, int slot = 0)
{
    k_creduce<NV><<<CRG, CRT, 0, s>>>(ncoarse(M), f, M->w.partial);
    k_cfinish<NV><<<1, 32, 0, s>>>(M->w.partial, M->w.scal + slot);
    MGC_CUDA(cudaGetLastError());
    count(2, (double)ncoarse(M) * 8.0 * 2);
    return MGC_OK;
}

template <class F>
int cmap(mgc_mg_s *M, F f, cudaStream_t s)
{
    k_cmap<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), f);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)ncoarse(M) * 8.0 * 3);
    return MGC_OK;
}

int fnorm2(mgc_mg_s *M, const float4 *v, double *out, cudaStream_t s)
{
    k_fnorm2<<<FNG, CRT, 0, s>>>(fine4(M), v, M->w.partial);
    k_cfinish<1><<<1, 32, 0, s>>>(M->w.partial, M->w.scal, FNG);
    MGC_CUDA(cudaGetLastError());
    count(2, (double)fine32_bytes(M));
    return read_scalars(M, 1, out, s);
}

// fraction of the fine sites a coarse-operator column's field occupies: all
// for the local entry k = 0, one face layer of each aggregate for k >= 1
static double field_fraction(const MgGeom &m, int k)
{
    if (k == 0) return 1.0;
    const int mu = (k - 1) / 2;
    return 1.0 / (double)(m.ratio[mu] << m.g.lb[mu]);
}

int do_restrict(mgc_mg_s *M, const float4 *v, float2 *u, cudaStream_t s, int k = 0, int colq = -1)
{
    dim3 grid((M->m.Vc + RWARPS - 1) / RWARPS, (M->m.nvec + CHUNK - 1) / CHUNK);
    k_restrict<1><<<grid, RWARPS * 32, 0, s>>>(M->m, M->w.W, v, nullptr, u, M->w.Dc, k, colq);
    MGC_CUDA(cudaGetLastError());
    const double frac = colq >= 0 ? field_fraction(M->m, k) : 1.0;
    count(1, (double)fine32_bytes(M) * (M->m.nvec + grid.y) * frac);
    return MGC_OK;
}

// columns colq and colq + 1 of coarse stencil entry k from their fields v, v2
// in one pass over the basis
int do_restrict2(mgc_mg_s *M, const float4 *v, const float4 *v2, cudaStream_t s, int k, int colq)
{
    dim3 grid((M->m.Vc + RWARPS - 1) / RWARPS, (M->m.nvec + CHUNK - 1) / CHUNK);
    k_restrict<2><<<grid, RWARPS * 32, 0, s>>>(M->m, M->w.W, v, v2, nullptr, M->w.Dc, k, colq);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)fine32_bytes(M) * (M->m.nvec + 2 * grid.y) * field_fraction(M->m, k));
    return MGC_OK;
}

int do_prolong(mgc_mg_s *M, const float2 *u, float4 *v, int add, cudaStream_t s)
{
    k_prolong<<<grid_for(M->m.g.V, 256), 256, 0, s>>>(M->m, M->w.W, u, v, add);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)fine32_bytes(M) * (M->m.nvec + 1 + add));
    return MGC_OK;
}

int coarse_apply(mgc_mg_s *M, const float2 *u, float2 *out, cudaStream_t s)
{
    k_coarse_apply<<<M->m.Vc, (M->m.n2 + 31) / 32 * 32, 0, s>>>(M->m, M->w.Dc, u, out);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)M->m.Vc * 9 * M->m.n2 * M->m.n2 * 8.0 + (double)ncoarse(M) * 16.0);
    return MGC_OK;
}

// W from Vraw: copy, block Gram-Schmidt; then the coarse stencil column by column
int build(mgc_mg_s *M, cudaStream_t s)
{
    MgWork &w = M->w;
    const Geom &g = M->m.g;
    const mgc_clover_s *op = M->op;
    MGC_CUDA(cudaMemcpyAsync(w.W, w.Vraw, fine32_bytes(M) * M->m.nvec, cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemsetAsync(w.dbad, 0, sizeof(int), s));
    k_block_gs<<<dim3(M->m.Vc, 2), 1 << g.lvb, 0, s>>>(M->m, w.W, w.dbad);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)fine32_bytes(M) * M->m.nvec * M->m.nvec);
    int bad = 0;
    MGC_CUDA(cudaMemcpyAsync(&bad, w.dbad, sizeof(int), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    if (bad) return fail(MGC_ERR_BREAKDOWN, "multigrid: null vectors linearly dependent on an aggregate");
    const Clover32 C{(float4 *)op->C32, g.lvb};
    const float kappa = (float)op->kappa;
    const size_t fs = (size_t)g.V * 6;
    auto field = [&](int chi, int i, int k, float4 *H) -> int {
        const Chiral32 p{Spinor32{w.W + i * fs, g.lvb}, chi};
        if (op->gauge->compress == 12)
            k_stencil_field<<<grid_for(g.V, 256), 256, 0, s>>>(M->m, p, Gauge32x12{(float4 *)op->gauge->U32, g.lvb},
                                                               C, kappa, k, H);
        else
            k_stencil_field<<<grid_for(g.V, 256), 256, 0, s>>>(M->m, p, Gauge32x18{(float2 *)op->gauge->U32, g.lvb},
                                                               C, kappa, k, H);
        MGC_CUDA(cudaGetLastError());
        count(1, (double)g.V * field_fraction(M->m, k) *
                     (96.0 * 2 + links_site_bytes(32, op->gauge->compress) + clover_site_bytes(32)));
        return MGC_OK;
    };
    // columns (chi, i) and (chi, i + 1) of each entry share a pass over the basis
    for (int chi = 0; chi < 2; ++chi)
        for (int i = 0; i < M->m.nvec; i += 2)
            for (int k = 0; k < 9; ++k) {
                const int col = chi * M->m.nvec + i;
                MGC_TRY(field(chi, i, k, w.f0));
                if (i + 1 < M->m.nvec) {
                    MGC_TRY(field(chi, i + 1, k, w.f1));
                    MGC_TRY(do_restrict2(M, w.f0, w.f1, s, k, col));
                } else {
                    MGC_TRY(do_restrict(M, w.f0, nullptr, s, k, col));
                }
            }
    M->ready = 1;
    return MGC_OK;
}

// BiCGStab on D_c x = b (coarse FP32 vectors) to tol or maxit.  The scalars
// stay on the device (the update kernels form alpha, omega and beta from
// them); the host reads ||r||^2 once per iteration to stop.
int coarse_solve(mgc_mg_s *M, const float2 *b, float2 *x, double tol, int maxit, int *iters, cudaStream_t s)
{
    MgWork &w = M->w;
    const int n = ncoarse(M);
    float2 *r = w.cr, *r0 = w.cr0, *p = w.cp, *v = w.cv, *sv = w.cs, *t = w.ct;
    const double *sc = w.scal;
    MGC_CUDA(cudaMemcpyAsync(r, b, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemcpyAsync(r0, b, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemcpyAsync(p, b, n * sizeof(float2), cudaMemcpyDeviceToDevice, s));
    MGC_CUDA(cudaMemsetAsync(x, 0, n * sizeof(float2), s));
    // ||b||^2 into CS_RR, rho = <r0, r> into CS_RHO (two slots after it)
    MGC_TRY(creduce<3>(M, [=] __device__(int e, double *acc) {
        const float2 q = r[e];
        acc[0] += (double)q.x * q.x + (double)q.y * q.y;
        ddot(acc + 1, r0[e], q);
    }, s, CS_RR));
    MGC_CUDA(cudaMemcpyAsync(w.scal + CS_RHO, w.scal + CS_RHO1, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    double h;
    MGC_CUDA(cudaMemcpyAsync(w.hscal, w.scal + CS_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    const double bn = std::sqrt(w.hscal[0]);
    int it = 0;
    if (bn == 0.0) {
        *iters = 0;
        return MGC_OK;
    }
    while (it < maxit) {
        MGC_TRY(coarse_apply(M, p, v, s));
        MGC_TRY(creduce<2>(M, [=] __device__(int e, double *acc) { ddot(acc, r0[e], v[e]); }, s, CS_R0V));
        MGC_TRY(cmap(M, [=] __device__(int e) {
            const float2 a = tof(cs_alpha(sc));
            sv[e] = cmad(make_float2(-a.x, -a.y), v[e], r[e]);
        }, s));
        MGC_TRY(coarse_apply(M, sv, t, s));
        MGC_TRY(creduce<3>(M, [=] __device__(int e, double *acc) {
            const float2 q = t[e];
            acc[0] += (double)q.x * q.x + (double)q.y * q.y;
            ddot(acc + 1, q, sv[e]);
        }, s, CS_TT));
        MGC_TRY(creduce<3>(M, [=] __device__(int e, double *acc) {
            const float2 a = tof(cs_alpha(sc)), o = tof(cs_omega(sc));
            x[e] = cmad(o, sv[e], cmad(a, p[e], x[e]));
            const float2 q = cmad(make_float2(-o.x, -o.y), t[e], sv[e]);
            r[e] = q;
            acc[0] += (double)q.x * q.x + (double)q.y * q.y;
            ddot(acc + 1, r0[e], q);
        }, s, CS_RR));
        MGC_CUDA(cudaMemcpyAsync(w.hscal, w.scal + CS_RR, sizeof(double), cudaMemcpyDeviceToHost, s));
        MGC_CUDA(cudaStreamSynchronize(s));
        h = w.hscal[0];
        ++it;
        if (!std::isfinite(h)) return fail(MGC_ERR_BREAKDOWN, "coarse BiCGStab: non-finite residual");
        if (std::sqrt(h) <= tol * bn) break;
        // p = r + beta (p - omega v), beta = (rho1 / rho)(alpha / omega); then rho = rho1
        MGC_TRY(cmap(M, [=] __device__(int e) {
            const double2 om = cs_omega(sc);
            const double2 beta = zmul(zdiv(ldz(sc + CS_RHO1), ldz(sc + CS_RHO)), zdiv(cs_alpha(sc), om));
            const float2 o = tof(om), bt = tof(beta);
            const float2 q = cmad(make_float2(-o.x, -o.y), v[e], p[e]);
            p[e] = cmad(bt, q, r[e]);
        }, s));
        MGC_CUDA(cudaMemcpyAsync(w.scal + CS_RHO, w.scal + CS_RHO1, 2 * sizeof(double), cudaMemcpyDeviceToDevice, s));
    }
    *iters = it;
    return MGC_OK;
}

// out = the SAP for A applied to in (FP32 fields), at the smoother precision
int smooth_A(mgc_mg_s *M, const mgc_mg_params *p, const float4 *in, float4 *out, cudaStream_t s)
{
    const Geom &g = M->m.g;
    if (p->smoother_prec == 32) {
        MGC_CUDA(cudaMemsetAsync(out, 0, fine32_bytes(M), s));
        return launch_sap_A(M->op, 32, in, out, 1, p->n_cy, p->n_jacobi, 1, s);
    }
    MGC_TRY(launch_convert(g, 1, 32, in, 16, M->w.l16a, s));
    MGC_CUDA(cudaMemsetAsync(M->w.l16b, 0, spinor_bytes(g, 16, 1), s));
    MGC_TRY(launch_sap_A(M->op, 16, M->w.l16a, M->w.l16b, 1, p->n_cy, p->n_jacobi, 1, s));
    return launch_convert(g, 1, 16, M->w.l16b, 32, out, s);
}

}  // namespace

// x = the two-level preconditioner applied to v (FP32 fine fields; v, x distinct from f0..f2)
int mg_precond32(mgc_mg_s *M, const mgc_mg_params *p, const float4 *v, float4 *x, cudaStream_t s)
{
    MgWork &w = M->w;
    const long long n4 = fine4(M);
    int it = 0;
    MGC_TRY(do_restrict(M, v, w.cb, s));
    MGC_TRY(coarse_solve(M, w.cb, w.cx, p->coarse_tol, p->coarse_maxit, &it, s));
    MGC_TRY(do_prolong(M, w.cx, x, 0, s));
    MGC_TRY(launch_dirac(M->op, 32, false, x, w.f0, 1, s));
    k_fsub<<<fgrid(n4, 256), 256, 0, s>>>(n4, v, w.f0, w.f0);
    MGC_CUDA(cudaGetLastError());
    count(1, 3.0 * fine32_bytes(M));
    MGC_TRY(launch_clover_apply(M->op, 32, true, w.f0, w.f1, 1, s));
    MGC_TRY(smooth_A(M, p, w.f1, w.f2, s));
    k_fadd<<<fgrid(n4, 256), 256, 0, s>>>(n4, w.f2, x);
    MGC_CUDA(cudaGetLastError());
    count(1, 3.0 * fine32_bytes(M));
    return MGC_OK;
}

// z = B v for FP64 packed fields: v / ||v|| to FP32, B, back scaled by ||v||
int mg_precond64(mgc_mg_s *M, const mgc_mg_params *p, const double2 *v, double2 *z, double vnorm, cudaStream_t s)
{
    const Geom &g = M->m.g;
    if (vnorm == 0.0) {
        MGC_CUDA(cudaMemsetAsync(z, 0, spinor_bytes(g, 64, 1), s));
        return MGC_OK;
    }
    MGC_TRY(launch_scale_to32(g, v, M->w.f3, 1.0 / vnorm, s));
    MGC_TRY(mg_precond32(M, p, M->w.f3, M->w.f4, s));
    MGC_CUDA(cudaMemsetAsync(z, 0, spinor_bytes(g, 64, 1), s));
    return launch_axpy_from32(g, z, M->w.f4, vnorm, 0.0, s);
}

mgc_clover_s *mg_operator(mgc_mg_s *M) { return M->op; }
int mg_ready(const mgc_mg_s *M) { return M->ready; }

}  // namespace mgc

// ------------------------------------------------------------------ C ABI
extern "C" {

void mgc_mg_params_default(mgc_mg_params *p)
{
    if (!p) return;
    p->n_cy = 2;
    p->n_jacobi = 4;
    p->smoother_prec = 32;
    p->coarse_tol = 5e-2;
    p->coarse_maxit = 100;
    p->n_adapt = 4;
}

static void mg_free(mgc_mg_s *M)
{
    MgWork &w = M->w;
    void *ptrs[] = {w.W, w.Vraw, w.Dc, w.cb, w.cx, w.cr, w.cr0, w.cp, w.cv, w.cs, w.ct, w.f0, w.f1, w.f2, w.f3,
                    w.f4, w.l16a, w.l16b, w.d0, w.d1, w.partial, w.scal, w.dbad};
    for (void *q : ptrs)
        if (q) cudaFree(q);
    if (w.hscal) cudaFreeHost(w.hscal);
    delete M;
}

int mgc_mg_create(mgc_clover_t op, const int agg[4], int nvec, mgc_mg_t *out)
{
    if (!op || !agg || !out) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    *out = nullptr;
    if (nvec < 1 || nvec > MGC_MG_MAX_NVEC) return fail(MGC_ERR_INVALID_ARG, "nvec must be in 1..32");
    if (!has_prec(op->gauge, 32)) return fail(MGC_ERR_INVALID_ARG, "the multigrid needs an operator with an FP32 copy");
    const Geom &g = op->gauge->lat->g;
    if ((1 << g.lvb) > 256) return fail(MGC_ERR_UNSUPPORTED_SHAPE, "SAP domains are limited to 256 sites");
    mgc_mg_s *M = new mgc_mg_s();
    M->op = op;
    M->m.g = g;
    M->m.nvec = nvec;
    M->m.n2 = 2 * nvec;
    M->m.da = 1;
    M->m.Vc = 1;
    for (int mu = 0; mu < 4; ++mu) {
        const int B = 1 << g.lb[mu];
        if (agg[mu] < B || agg[mu] % B != 0 || g.L[mu] % agg[mu] != 0) {
            delete M;
            return fail(MGC_ERR_UNSUPPORTED_SHAPE,
                        "aggregate extents must be multiples of the SAP domain and divide the lattice");
        }
        M->m.ratio[mu] = agg[mu] / B;
        M->m.Lc[mu] = g.L[mu] / agg[mu];
        M->m.da *= M->m.ratio[mu];
        M->m.Vc *= M->m.Lc[mu];
    }
    MgWork &w = M->w;
    const size_t f32 = (size_t)g.V * 96, f64 = (size_t)g.V * 192;
    const size_t nc = (size_t)M->m.Vc * M->m.n2 * sizeof(float2);
    bool okm = cudaMalloc(&w.W, f32 * nvec) == cudaSuccess && cudaMalloc(&w.Vraw, f32 * nvec) == cudaSuccess &&
               cudaMalloc(&w.Dc, (size_t)M->m.Vc * 9 * M->m.n2 * M->m.n2 * sizeof(float2)) == cudaSuccess;
    float2 **cv[] = {&w.cb, &w.cx, &w.cr, &w.cr0, &w.cp, &w.cv, &w.cs, &w.ct};
    for (auto q : cv) okm = okm && cudaMalloc(q, nc) == cudaSuccess;
    float4 **fv[] = {&w.f0, &w.f1, &w.f2, &w.f3, &w.f4};
    for (auto q : fv) okm = okm && cudaMalloc(q, f32) == cudaSuccess;
    okm = okm && cudaMalloc(&w.d0, f64) == cudaSuccess && cudaMalloc(&w.d1, f64) == cudaSuccess;
    if (op->gauge->prec == 16)
        okm = okm && cudaMalloc(&w.l16a, spinor_bytes(g, 16, 1)) == cudaSuccess &&
              cudaMalloc(&w.l16b, spinor_bytes(g, 16, 1)) == cudaSuccess;
    okm = okm && cudaMalloc(&w.partial, CRG * 4 * sizeof(double)) == cudaSuccess &&
          cudaMalloc(&w.scal, 16 * sizeof(double)) == cudaSuccess && cudaMalloc(&w.dbad, sizeof(int)) == cudaSuccess &&
          cudaMallocHost(&w.hscal, 16 * sizeof(double)) == cudaSuccess;
    if (!okm) {
        cudaGetLastError();
        mg_free(M);
        return fail(MGC_ERR_CUDA, "multigrid: out of device memory");
    }
    *out = M;
    return ok();
}

int mgc_mg_destroy(mgc_mg_t M)
{
    if (!M) return MGC_OK;
    cudaDeviceSynchronize();
    mg_free(M);
    return ok();
}

long long mgc_mg_coarse_volume(mgc_mg_t M) { return M ? M->m.Vc : 0; }

static int check_mgp(const mgc_mg_s *M, const mgc_mg_params *p)
{
    if (!p) return fail(MGC_ERR_INVALID_ARG, "NULL multigrid parameters");
    if (p->smoother_prec != 32 && p->smoother_prec != 16)
        return fail(MGC_ERR_INVALID_ARG, "multigrid smoother_prec must be 32 or 16");
    if (!has_prec(M->op->gauge, p->smoother_prec))
        return fail(MGC_ERR_INVALID_ARG, "no copy of the operator at the smoother precision");
    if (p->n_cy < 0 || p->n_jacobi < 0 || p->coarse_maxit < 1 || !(p->coarse_tol > 0) || p->n_adapt < 0)
        return fail(MGC_ERR_INVALID_ARG, "bad multigrid parameters");
    return MGC_OK;
}

// FP64 canonical fine field -> FP32 packed
static int canon_to32(mgc_mg_s *M, const double *in, float4 *out, cudaStream_t s)
{
    MGC_TRY(launch_pack(M->m.g, 64, 1, in, M->w.d0, s));
    return launch_scale_to32(M->m.g, M->w.d0, out, 1.0, s);
}

static int f32_to_canon(mgc_mg_s *M, const float4 *in, double *out, cudaStream_t s)
{
    MGC_CUDA(cudaMemsetAsync(M->w.d0, 0, (size_t)M->m.g.V * 192, s));
    MGC_TRY(launch_axpy_from32(M->m.g, M->w.d0, in, 1.0, 0.0, s));
    return launch_unpack(M->m.g, 64, 1, M->w.d0, out, s);
}

int mgc_mg_set_vectors(mgc_mg_t M, const double *V, void *stream)
{
    if (!M || !V) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fs = (size_t)M->m.g.V * 6;
    for (int i = 0; i < M->m.nvec; ++i) MGC_TRY(canon_to32(M, V + (size_t)i * M->m.g.V * 24, M->w.Vraw + i * fs, s));
    return build(M, s);
}

int mgc_mg_setup(mgc_mg_t M, const double *eta, const mgc_mg_params *p, void *stream)
{
    if (!M || !eta) return fail(MGC_ERR_INVALID_ARG, "NULL argument");
    MGC_TRY(check_mgp(M, p));
    cudaStream_t s = (cudaStream_t)stream;
    const Geom &g = M->m.g;
    const size_t fs = (size_t)g.V * 6;
    MgWork &w = M->w;
    // V_i = M_SAP(C^-1 eta_i)
    for (int i = 0; i < M->m.nvec; ++i) {
        MGC_TRY(launch_pack(g, 64, 1, eta + (size_t)i * g.V * 24, w.d0, s));
        MGC_TRY(launch_clover_apply(M->op, 64, true, w.d0, w.d1, 1, s));
        MGC_TRY(launch_scale_to32(g, w.d1, w.f3, 1.0, s));
        MGC_TRY(smooth_A(M, p, w.f3, w.Vraw + i * fs, s));
    }
    MGC_TRY(build(M, s));
    for (int pass = 0; pass < p->n_adapt; ++pass) {
        for (int i = 0; i < M->m.nvec; ++i) {
            float4 *vi = w.Vraw + i * fs;
            MGC_TRY(mg_precond32(M, p, vi, w.f4, s));
            double n2 = 0;
            MGC_TRY(fnorm2(M, w.f4, &n2, s));
            if (!(n2 > 0) || !std::isfinite(n2)) return fail(MGC_ERR_BREAKDOWN, "multigrid setup: zero vector");
            MGC_CUDA(cudaMemcpyAsync(vi, w.f4, fine32_bytes(M), cudaMemcpyDeviceToDevice, s));
            k_fscale<<<fgrid(fine4(M), 256), 256, 0, s>>>(fine4(M), (float)(1.0 / std::sqrt(n2)), vi);
            MGC_CUDA(cudaGetLastError());
            count(1, 2.0 * fine32_bytes(M));
        }
        MGC_TRY(build(M, s));
    }
    MGC_CUDA(cudaStreamSynchronize(s));
    return check_device_status(M->op, s);
}

int mgc_mg_export(mgc_mg_t M, double *W, double *Dc, void *stream)
{
    if (!M || !M->ready) return fail(MGC_ERR_INVALID_ARG, "multigrid handle without a basis");
    cudaStream_t s = (cudaStream_t)stream;
    const size_t fs = (size_t)M->m.g.V * 6;
    if (W)
        for (int i = 0; i < M->m.nvec; ++i) MGC_TRY(f32_to_canon(M, M->w.W + i * fs, W + (size_t)i * M->m.g.V * 24, s));
    if (Dc) {
        const int nblk = M->m.Vc * 9;
        k_export_stencil<<<fgrid((long long)nblk * M->m.n2 * M->m.n2, 256), 256, 0, s>>>(nblk, M->m.n2, M->w.Dc,
                                                                                       (double2 *)Dc);
        MGC_CUDA(cudaGetLastError());
    }
    return ok();
}

int mgc_mg_restrict(mgc_mg_t M, const double *v, double *u, void *stream)
{
    if (!M || !M->ready || !v || !u) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    MGC_TRY(canon_to32(M, v, M->w.f3, s));
    MGC_TRY(do_restrict(M, M->w.f3, M->w.cb, s));
    k_c32_to64<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), M->w.cb, (double2 *)u);
    MGC_CUDA(cudaGetLastError());
    return ok();
}

int mgc_mg_prolong(mgc_mg_t M, const double *u, double *v, void *stream)
{
    if (!M || !M->ready || !v || !u) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    k_c64_to32<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), (const double2 *)u, M->w.cb);
    MGC_CUDA(cudaGetLastError());
    MGC_TRY(do_prolong(M, M->w.cb, M->w.f3, 0, s));
    return f32_to_canon(M, M->w.f3, v, s);
}

int mgc_mg_coarse_apply(mgc_mg_t M, const double *u, double *out, void *stream)
{
    if (!M || !M->ready || !u || !out) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    k_c64_to32<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), (const double2 *)u, M->w.cb);
    MGC_TRY(coarse_apply(M, M->w.cb, M->w.cx, s));
    k_c32_to64<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), M->w.cx, (double2 *)out);
    MGC_CUDA(cudaGetLastError());
    return ok();
}

int mgc_mg_coarse_solve(mgc_mg_t M, const double *b, double *x, double tol, int maxit, int *iters, void *stream)
{
    if (!M || !M->ready || !b || !x || !iters || !(tol > 0) || maxit < 1) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    cudaStream_t s = (cudaStream_t)stream;
    // the coarse solve works in cx/cr..; the right-hand side goes to f-free coarse storage cb
    k_c64_to32<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), (const double2 *)b, M->w.cb);
    MGC_CUDA(cudaGetLastError());
    MGC_TRY(coarse_solve(M, M->w.cb, M->w.cx, tol, maxit, iters, s));
    k_c32_to64<<<fgrid(ncoarse(M), 256), 256, 0, s>>>(ncoarse(M), M->w.cx, (double2 *)x);
    MGC_CUDA(cudaGetLastError());
    MGC_CUDA(cudaStreamSynchronize(s));
    return ok();
}

int mgc_mg_precond(mgc_mg_t M, const double *v, double *x, const mgc_mg_params *p, void *stream)
{
    if (!M || !M->ready || !v || !x) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    MGC_TRY(check_mgp(M, p));
    cudaStream_t s = (cudaStream_t)stream;
    MGC_TRY(canon_to32(M, v, M->w.f3, s));
    MGC_TRY(mg_precond32(M, p, M->w.f3, M->w.f4, s));
    MGC_TRY(f32_to_canon(M, M->w.f4, x, s));
    MGC_CUDA(cudaStreamSynchronize(s));
    return check_device_status(M->op, s);
}

int mgc_mg_solve(mgc_mg_t M, const double *b, double *x, const mgc_solve_params *p, const mgc_mg_params *mp,
                 mgc_solve_info *info, void *stream)
{
    if (!M || !M->ready || !b || !x || !p || !info) return fail(MGC_ERR_INVALID_ARG, "bad argument");
    MGC_TRY(check_mgp(M, mp));
    return mgc::mg_solve(M, b, x, p, mp, info, (cudaStream_t)stream);
}

}  // extern "C"
