// The Wilson hopping sum at one site, Eq. (1):
//   acc += sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)]
// (projector signs swapped for D^dagger), with the t-boundary sign on the hops
// that wrap in t.  Each hop is projected to a two-spin half spinor before the
// SU(3) multiply, so a hop costs two colour mat-vecs instead of four.
#pragma once

#include "mgc_device.cuh"

namespace mgc {

// h = P psi(j) for the projector 1 + SGN gamma_mu, with the t-boundary sign
template <int MU, int SGN, class SP, typename T>
__device__ __forceinline__ void load_project(const SP &in, int j, bool flip, Cx<T> h[6])
{
    Cx<T> s[12];
    in.load(j, s);
    project<MU, SGN>(s, h);
    if (flip) negate6(h);
}

// FP16 spinors: project the stored halves and apply the per-site scale (and
// the boundary sign) to the six projected components only
template <int MU, int SGN>
__device__ __forceinline__ void load_project(const Spinor16 &in, int j, bool flip, Cx<float> h[6])
{
    Cx<float> s[12];
    in.load_raw(j, s);
    project<MU, SGN>(s, h);
    const float sc = flip ? -in.scale_of(j) : in.scale_of(j);
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = sc * h[k];
}

// ---- the operator kernels' form: every hop is accumulated with a real
// coefficient by fused multiply-adds, the coefficient carrying -kappa, the
// boundary sign and (FP16 spinors) the neighbour's per-site scale, so no
// separate scaling or kappa multiplication is left

// h = P psi(j) unscaled; returns the factor that restores psi's scale
template <int MU, int SGN, class SP, typename T>
__device__ __forceinline__ T load_project_s(const SP &in, int j, Cx<T> h[6])
{
    Cx<T> s[12];
    in.load(j, s);
    project<MU, SGN>(s, h);
    return T(1);
}
template <int MU, int SGN>
__device__ __forceinline__ float load_project_s(const Spinor16 &in, int j, Cx<float> h[6])
{
    Cx<float> s[12];
    in.load_raw(j, s);
    project<MU, SGN>(s, h);
    return in.scale_of(j);
}

// psi(i) unscaled and its scale factor
template <class SP, typename T>
__device__ __forceinline__ T load_s(const SP &in, int i, Cx<T> psi[12])
{
    in.load(i, psi);
    return T(1);
}
__device__ __forceinline__ float load_s(const Spinor16 &in, int i, Cx<float> psi[12])
{
    in.load_raw(i, psi);
    return in.scale_of(i);
}

// out = C(i) psi unscaled; returns the clover's scale factor
template <class CL, typename T>
__device__ __forceinline__ T clover_site_s(const CL &C, int i, const Cx<T> psi[12], Cx<T> out[12])
{
    T cl[72];
    C.load(i, cl);
    clover_mul(cl, psi, out);
    return T(1);
}
__device__ __forceinline__ float clover_site_s(const Clover16 &C, int i, const Cx<float> psi[12], Cx<float> out[12])
{
    float cl[72];
    const float sc = C.load_raw(i, cl);
    clover_mul(cl, psi, out);
    return sc;
}

// acc += coef * (the four-spinor reconstructed from w)
template <int MU, int SGN, typename T>
__device__ __forceinline__ void reconstruct_fma(Cx<T> acc[12], const Cx<T> w[6], T coef)
{
    const T lo = (MU == 3 ? (SGN > 0 ? -coef : coef) : (SGN > 0 ? coef : -coef));
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = Cx<T>{fma(coef, w[c].r, acc[c].r), fma(coef, w[c].i, acc[c].i)};
        acc[3 + c] = Cx<T>{fma(coef, w[3 + c].r, acc[3 + c].r), fma(coef, w[3 + c].i, acc[3 + c].i)};
        Cx<T> o0, o1;
        if (MU == 3) {
            o0 = w[c];
            o1 = w[3 + c];
        } else {
            isigma<MU>(w[c], w[3 + c], o0, o1);
        }
        acc[6 + c] = Cx<T>{fma(lo, o0.r, acc[6 + c].r), fma(lo, o0.i, acc[6 + c].i)};
        acc[9 + c] = Cx<T>{fma(lo, o1.r, acc[9 + c].r), fma(lo, o1.i, acc[9 + c].i)};
    }
}

// acc += mk * (the two hops along MU), mk = -kappa
template <int MU, bool DAG, class SP, class GA, typename T>
__device__ __forceinline__ void hop_dir_k(const Geom &g, const int c[4], int i, const SP &in, const GA &U, T mk,
                                          Cx<T> acc[12])
{
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    bool wr;
    Cx<T> h[6], w[6], u[9];
    int j = neighbour(g, c, MU, +1, &wr);
    T coef = mk * load_project_s<MU, SF>(in, j, h);
    if (MU == 3 && wr && g.tbc < 0) coef = -coef;
    U.load(i, MU, u);
    su3_mul(u, h, w);
    reconstruct_fma<MU, SF>(acc, w, coef);

    j = neighbour(g, c, MU, -1, &wr);
    coef = mk * load_project_s<MU, SB>(in, j, h);
    if (MU == 3 && wr && g.tbc < 0) coef = -coef;
    U.load(j, MU, u);
    su3_dag_mul(u, h, w);
    reconstruct_fma<MU, SB>(acc, w, coef);
}

template <int MU, bool DAG, class SP, class GA, typename T>
__device__ __forceinline__ void hop_dir(const Geom &g, const int c[4], int i, const SP &in, const GA &U,
                                        Cx<T> acc[12])
{
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_mu
    constexpr int SB = -SF;            // backward projector 1 + SB gamma_mu
    bool wr;
    Cx<T> h[6], w[6], u[9];
    int j = neighbour(g, c, MU, +1, &wr);
    load_project<MU, SF>(in, j, MU == 3 && wr && g.tbc < 0, h);
    U.load(i, MU, u);
    su3_mul(u, h, w);
    reconstruct_add<MU, SF>(acc, w);

    j = neighbour(g, c, MU, -1, &wr);
    load_project<MU, SB>(in, j, MU == 3 && wr && g.tbc < 0, h);
    U.load(j, MU, u);
    su3_dag_mul(u, h, w);
    reconstruct_add<MU, SB>(acc, w);
}

template <bool DAG, class SP, class GA, typename T>
__device__ __forceinline__ void hop_site(const Geom &g, const int c[4], int i, const SP &in, const GA &U,
                                         Cx<T> acc[12])
{
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = Cx<T>{0, 0};
    hop_dir<0, DAG>(g, c, i, in, U, acc);
    hop_dir<1, DAG>(g, c, i, in, U, acc);
    hop_dir<2, DAG>(g, c, i, in, U, acc);
    hop_dir<3, DAG>(g, c, i, in, U, acc);
}

// The hopping sums of RB right-hand sides at one site in the operator
// kernels' form (coefficient mk = -kappa), each link loaded once and applied
// to all of them; only the first nr (<= RB) are computed.
template <int MU, bool DAG, int RB, class SP, class GA, typename T>
__device__ __forceinline__ void hop_dir_multi(const Geom &g, const int c[4], int i, const SP (&in)[RB], int nr,
                                              const GA &U, T mk, Cx<T> (&acc)[RB][12])
{
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    bool wr;
    Cx<T> h[6], w[6], u[9];
    int j = neighbour(g, c, MU, +1, &wr);
    bool flip = MU == 3 && wr && g.tbc < 0;
    U.load(i, MU, u);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            T coef = mk * load_project_s<MU, SF>(in[q], j, h);
            if (flip) coef = -coef;
            su3_mul(u, h, w);
            reconstruct_fma<MU, SF>(acc[q], w, coef);
        }
    j = neighbour(g, c, MU, -1, &wr);
    flip = MU == 3 && wr && g.tbc < 0;
    U.load(j, MU, u);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            T coef = mk * load_project_s<MU, SB>(in[q], j, h);
            if (flip) coef = -coef;
            su3_dag_mul(u, h, w);
            reconstruct_fma<MU, SB>(acc[q], w, coef);
        }
}

template <bool DAG, int RB, class SP, class GA, typename T>
__device__ __forceinline__ void hop_site_multi(const Geom &g, const int c[4], int i, const SP (&in)[RB], int nr,
                                               const GA &U, T mk, Cx<T> (&acc)[RB][12])
{
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[q][k] = Cx<T>{0, 0};
    hop_dir_multi<0, DAG>(g, c, i, in, nr, U, mk, acc);
    hop_dir_multi<1, DAG>(g, c, i, in, nr, U, mk, acc);
    hop_dir_multi<2, DAG>(g, c, i, in, nr, U, mk, acc);
    hop_dir_multi<3, DAG>(g, c, i, in, nr, U, mk, acc);
}

// ---- the FP64 operator's form, where every FP64 instruction counts (GB300
// issues FP64 at 1/64 of the FP32 rate): the two hops along MU are combined
// before they reach the accumulator.  With w_f = U_mu(x) h_f and
// w_b = U_mu(x-mu)^+ h_b, and the two projector signs opposite, the upper
// spins receive c (w_f + g w_b) and the lower spins sig c P(w_f - g w_b),
// where P is the isigma map of the projection (identity for mu = t), sig its
// sign, c the forward hop's coefficient and g = +-1 the ratio of the backward
// hop's coefficient to it (-1 only where exactly one of the two hops wraps an
// antiperiodic t boundary).  s = w_f + g w_b comes out of the backward mat-vec
// accumulating onto w_f, and w_f - g w_b = 2 w_f - s, so a pair of hops takes
// 204 FP64 instructions instead of 216.

// s = w + U^dagger h (two colour vectors)
template <typename T>
__device__ __forceinline__ void su3_dag_mul_acc(const Cx<T> u[9], const Cx<T> h[6], const Cx<T> w[6], Cx<T> s[6])
{
#pragma unroll
    for (int q = 0; q < 2; ++q)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Cx<T> acc = cjfma(u[a], h[3 * q], w[3 * q + a]);
            acc = cjfma(u[3 + a], h[3 * q + 1], acc);
            acc = cjfma(u[6 + a], h[3 * q + 2], acc);
            s[3 * q + a] = acc;
        }
}

// acc += c (s on the upper spins) + sig c P(2 w - s) on the lower spins, for
// the forward projector 1 + SF gamma_mu
template <int MU, int SF, typename T>
__device__ __forceinline__ void reconstruct_pair(Cx<T> acc[12], const Cx<T> w[6], const Cx<T> s[6], T c)
{
    const T lo = (MU == 3 ? (SF > 0 ? -c : c) : (SF > 0 ? c : -c));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        acc[k] = Cx<T>{fma(c, s[k].r, acc[k].r), fma(c, s[k].i, acc[k].i)};
        acc[3 + k] = Cx<T>{fma(c, s[3 + k].r, acc[3 + k].r), fma(c, s[3 + k].i, acc[3 + k].i)};
        const Cx<T> d0 = {fma(T(2), w[k].r, -s[k].r), fma(T(2), w[k].i, -s[k].i)};
        const Cx<T> d1 = {fma(T(2), w[3 + k].r, -s[3 + k].r), fma(T(2), w[3 + k].i, -s[3 + k].i)};
        Cx<T> o0, o1;
        isigma<MU>(d0, d1, o0, o1);
        acc[6 + k] = Cx<T>{fma(lo, o0.r, acc[6 + k].r), fma(lo, o0.i, acc[6 + k].i)};
        acc[9 + k] = Cx<T>{fma(lo, o1.r, acc[9 + k].r), fma(lo, o1.i, acc[9 + k].i)};
    }
}

// acc[q] += mk * (the two hops along MU) for the first nr of RB right-hand
// sides, both links loaded once; RB = 1 is the single-RHS operator
template <int MU, bool DAG, int RB, class SP, class GA, typename T>
__device__ __forceinline__ void hop_pair_multi(const Geom &g, const int c[4], int i, const SP (&in)[RB], int nr,
                                               const GA &U, T mk, Cx<T> (&acc)[RB][12])
{
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    bool wf, wb;
    const int jf = neighbour(g, c, MU, +1, &wf);
    const int jb = neighbour(g, c, MU, -1, &wb);
    const bool ff = MU == 3 && wf && g.tbc < 0, fb = MU == 3 && wb && g.tbc < 0;
    const T cf = ff ? -mk : mk;
    Cx<T> uf[9], ub[9];
    U.load(i, MU, uf);
    U.load(jb, MU, ub);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            Cx<T> h[6], w[6], s[6];
            load_project_s<MU, SF>(in[q], jf, h);
            su3_mul(uf, h, w);
            load_project_s<MU, SB>(in[q], jb, h);
            if (ff != fb) negate6(h);
            su3_dag_mul_acc(ub, h, w, s);
            reconstruct_pair<MU, SF>(acc[q], w, s, cf);
        }
}

// out += C in for the packed clover c[72] (the accumulating form of clover_mul)
template <typename T>
__device__ __forceinline__ void clover_mul_acc(const T c[72], const Cx<T> in[12], Cx<T> out[12])
{
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        const T *d = c + 36 * chi;
        const Cx<T> *v = in + 6 * chi;
        Cx<T> *o = out + 6 * chi;
#pragma unroll
        for (int a = 0; a < 6; ++a) o[a] = Cx<T>{fma(d[a], v[a].r, o[a].r), fma(d[a], v[a].i, o[a].i)};
        int k = 6;
#pragma unroll
        for (int a = 1; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < a; ++b) {
                const Cx<T> L = {d[k], d[k + 1]};
                k += 2;
                o[a] = cfma(L, v[b], o[a]);
                o[b] = cjfma(L, v[a], o[b]);
            }
    }
}

// (D psi)(x) for RB right-hand sides at FP64 (unit scales): the paired hops
// with -kappa as their coefficient, then C psi accumulated onto them
template <bool DAG, int RB, class SP, class GA, class CL, typename T>
__device__ __forceinline__ void dirac_site_pair(const Geom &g, const int c[4], int i, const SP (&in)[RB], int nr,
                                                const GA &U, const CL &C, T kappa, Cx<T> (&out)[RB][12])
{
    static_assert(sizeof(T) == 8, "the paired form is the FP64 operator's");
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int k = 0; k < 12; ++k) out[q][k] = Cx<T>{0, 0};
    hop_pair_multi<0, DAG>(g, c, i, in, nr, U, -kappa, out);
    hop_pair_multi<1, DAG>(g, c, i, in, nr, U, -kappa, out);
    hop_pair_multi<2, DAG>(g, c, i, in, nr, U, -kappa, out);
    hop_pair_multi<3, DAG>(g, c, i, in, nr, U, -kappa, out);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            T cl[72];
            Cx<T> psi[12];
            C.load(i, cl);  // per right-hand side: 144 registers do not stay live across them
            in[q].load(i, psi);
            clover_mul_acc(cl, psi, out[q]);
        }
}

// out = C(i) psi
template <class CL, typename T>
__device__ __forceinline__ void clover_site(const CL &C, int i, const Cx<T> psi[12], Cx<T> out[12])
{
    T cl[72];
    C.load(i, cl);
    clover_mul(cl, psi, out);
}

// FP16 clover: multiply with the stored halves, scale the twelve results
__device__ __forceinline__ void clover_site(const Clover16 &C, int i, const Cx<float> psi[12], Cx<float> out[12])
{
    float cl[72];
    const float sc = C.load_raw(i, cl);
    clover_mul(cl, psi, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = sc * out[k];
}

// (D psi)(x) in the operator kernels' form: the hops accumulated with
// -kappa (and the spinor scales) as coefficients, then C psi added with the
// clover and spinor scales as one coefficient
template <bool DAG, class SP, class GA, class CL, typename T>
__device__ __forceinline__ void dirac_site_k(const Geom &g, const int c[4], int i, const SP &in, const GA &U,
                                             const CL &C, T kappa, Cx<T> out[12])
{
    Cx<T> acc[12], psi[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) acc[k] = Cx<T>{0, 0};
    hop_dir_k<0, DAG>(g, c, i, in, U, -kappa, acc);
    hop_dir_k<1, DAG>(g, c, i, in, U, -kappa, acc);
    hop_dir_k<2, DAG>(g, c, i, in, U, -kappa, acc);
    hop_dir_k<3, DAG>(g, c, i, in, U, -kappa, acc);
    const T sp = load_s(in, i, psi);
    const T sc = clover_site_s(C, i, psi, out) * sp;
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = Cx<T>{fma(sc, out[k].r, acc[k].r), fma(sc, out[k].i, acc[k].i)};
}

// (D psi)(x) = C(x) psi(x) - kappa * hop  at packed site i with coordinates c
template <bool DAG, class SP, class GA, class CL, typename T>
__device__ __forceinline__ void dirac_site(const Geom &g, const int c[4], int i, const SP &in, const GA &U,
                                           const CL &C, T kappa, Cx<T> out[12])
{
    Cx<T> acc[12], psi[12];
    hop_site<DAG>(g, c, i, in, U, acc);
    in.load(i, psi);
    clover_site(C, i, psi, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = Cx<T>{fma(-kappa, acc[k].r, out[k].r), fma(-kappa, acc[k].i, out[k].i)};
}

}  // namespace mgc
