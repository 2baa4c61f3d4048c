// The Wilson hopping sum at one site, Eq. (1):
//   acc += sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu) + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)]
// (projector signs swapped for D^dagger), with the t-boundary sign on the hops
// that wrap in t.  Each hop is projected to a two-spin half spinor before the
// SU(3) multiply, so a hop costs two colour mat-vecs instead of four.
#pragma once

#include "mgc_device.cuh"

namespace mgc {

template <int MU, bool DAG, class SP, class GA, typename T>
__device__ __forceinline__ void hop_dir(const Geom &g, const int c[4], int i, const SP &in, const GA &U,
                                        Cx<T> acc[12])
{
    constexpr int SF = DAG ? +1 : -1;  // forward projector 1 + SF gamma_mu
    constexpr int SB = -SF;            // backward projector 1 + SB gamma_mu
    bool wr;
    Cx<T> s[12], h[6], w[6], u[9];
    int j = neighbour(g, c, MU, +1, &wr);
    in.load(j, s);
    project<MU, SF>(s, h);
    if (MU == 3 && wr && g.tbc < 0) negate6(h);
    U.load(i, MU, u);
    su3_mul(u, h, w);
    reconstruct_add<MU, SF>(acc, w);

    j = neighbour(g, c, MU, -1, &wr);
    in.load(j, s);
    project<MU, SB>(s, h);
    if (MU == 3 && wr && g.tbc < 0) negate6(h);
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

// (D psi)(x) = C(x) psi(x) - kappa * hop  at packed site i with coordinates c
template <bool DAG, class SP, class GA, class CL, typename T>
__device__ __forceinline__ void dirac_site(const Geom &g, const int c[4], int i, const SP &in, const GA &U,
                                           const CL &C, T kappa, Cx<T> out[12])
{
    Cx<T> acc[12], psi[12];
    hop_site<DAG>(g, c, i, in, U, acc);
    in.load(i, psi);
    T cl[72];
    C.load(i, cl);
    clover_mul(cl, psi, out);
#pragma unroll
    for (int k = 0; k < 12; ++k) out[k] = Cx<T>{fma(-kappa, acc[k].r, out[k].r), fma(-kappa, acc[k].i, out[k].i)};
}

}  // namespace mgc
