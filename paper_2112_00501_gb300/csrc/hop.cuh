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

// The hopping sums of RB right-hand sides at one site, each link loaded once
// and applied to all of them; only the first nr (<= RB) are computed.
template <int MU, bool DAG, int RB, class SP, class GA, typename T>
__device__ __forceinline__ void hop_dir_multi(const Geom &g, const int c[4], int i, const SP (&in)[RB], int nr,
                                              const GA &U, Cx<T> (&acc)[RB][12])
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
            load_project<MU, SF>(in[q], j, flip, h);
            su3_mul(u, h, w);
            reconstruct_add<MU, SF>(acc[q], w);
        }
    j = neighbour(g, c, MU, -1, &wr);
    flip = MU == 3 && wr && g.tbc < 0;
    U.load(j, MU, u);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            load_project<MU, SB>(in[q], j, flip, h);
            su3_dag_mul(u, h, w);
            reconstruct_add<MU, SB>(acc[q], w);
        }
}

template <bool DAG, int RB, class SP, class GA, typename T>
__device__ __forceinline__ void hop_site_multi(const Geom &g, const int c[4], int i, const SP (&in)[RB], int nr,
                                               const GA &U, Cx<T> (&acc)[RB][12])
{
#pragma unroll
    for (int q = 0; q < RB; ++q)
#pragma unroll
        for (int k = 0; k < 12; ++k) acc[q][k] = Cx<T>{0, 0};
    hop_dir_multi<0, DAG>(g, c, i, in, nr, U, acc);
    hop_dir_multi<1, DAG>(g, c, i, in, nr, U, acc);
    hop_dir_multi<2, DAG>(g, c, i, in, nr, U, acc);
    hop_dir_multi<3, DAG>(g, c, i, in, nr, U, acc);
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
