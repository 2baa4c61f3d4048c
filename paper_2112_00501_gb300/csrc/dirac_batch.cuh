// The batched multi-RHS clover-Wilson operator (Eq. (1)): one launch for every
// right-hand side of every lattice of a batch.  Included by the three
// translation units that instantiate it (FP64, FP32, FP16 storage).
#pragma once

#include "hop.cuh"
#include "mgc_host.h"

namespace mgc {

namespace {
inline Spinor64 sp64(const Geom &g, const void *b) { return Spinor64{(double2 *)b, g.lvb}; }
inline Spinor32 sp32(const Geom &g, const void *b) { return Spinor32{(float4 *)b, g.lvb}; }
inline Spinor16 sp16(const Geom &g, const void *b, int nrhs)
{
    uint4 *d = (uint4 *)b;
    return Spinor16{d, (float *)(d + (size_t)nrhs * g.V * 3), g.lvb};
}
inline Clover16 cl16(const Geom &g, const mgc_clover_s *op) { return Clover16{(uint4 *)op->C16, op->C16_sc, g.lvb}; }

// One launch applies D to every right-hand side of every lattice of a batch.
// Each thread computes RB right-hand sides of one site and applies each link
// it loads to all of them.  Thread block b belongs to the first lattice k with
// b < end[k]; inside it, rhs_fast = 1 makes the blocks of one site block and
// consecutive right-hand-side groups adjacent (they share links in L2).
template <class SP, class GA, class CL> struct DiracBatch {
    int n;
    int rhs_fast;
    int end[MGC_BATCH_MAX];
    int nsb[MGC_BATCH_MAX];   // site blocks of one lattice
    int ngrp[MGC_BATCH_MAX];  // right-hand-side groups, ceil(nrhs / RB)
    int nrhs[MGC_BATCH_MAX];
    Geom g[MGC_BATCH_MAX];
    SP in[MGC_BATCH_MAX], out[MGC_BATCH_MAX];
    GA U[MGC_BATCH_MAX];
    CL C[MGC_BATCH_MAX];
    typename SP::Real kappa[MGC_BATCH_MAX];
};

// blocks per SM the register budget is set for: FP32 arithmetic with one RHS
// per thread fits 80 registers (three 256-thread blocks), two RHS 128 (two);
// four RHS and FP64 take one
template <int RB, class SP>
__host__ __device__ constexpr int dirac_batch_min_blocks()
{
    return sizeof(typename SP::Real) == 8 ? 1 : (RB == 1 ? 3 : (RB == 2 ? 2 : 1));
}

template <bool DAG, int LVB, int RB, class SP, class GA, class CL>
__global__ void __launch_bounds__(256, dirac_batch_min_blocks<RB, SP>()) k_dirac_batch(DiracBatch<SP, GA, CL> B)
{
    using T = typename SP::Real;
    int k = 0;
    while (k < B.n - 1 && (int)blockIdx.x >= B.end[k]) ++k;
    const int local = blockIdx.x - (k ? B.end[k - 1] : 0);
    int sb, grp;
    if (B.rhs_fast) {
        grp = local % B.ngrp[k];
        sb = local / B.ngrp[k];
    } else {
        sb = local % B.nsb[k];
        grp = local / B.nsb[k];
    }
    Geom gg = B.g[k];
    const int i = sb * blockDim.x + threadIdx.x;
    if (i >= gg.V) return;
    const int r0 = grp * RB;
    const int nr = min(RB, B.nrhs[k] - r0);
    GA Ug = B.U[k];
    CL Cg = B.C[k];
    SP base_in = B.in[k], base_out = B.out[k];
    if (LVB > 0) {
        gg.lvb = LVB;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LVB / 4;
        base_in.lvb = base_out.lvb = Ug.lvb = Cg.lvb = LVB;
    }
    SP src[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) src[q] = shift_rhs(base_in, r0 + (q < nr ? q : 0), gg.V);
    int c[4];
    site_coords(gg, i, c);
    Cx<T> acc[RB][12];
    const T kappa = B.kappa[k];
    if constexpr (sizeof(T) == 8) {
        // the single-RHS FP64 operator's arithmetic, right-hand side by right-hand side
        dirac_site_pair<DAG, RB>(gg, c, i, src, nr, Ug, Cg, kappa, acc);
#pragma unroll
        for (int q = 0; q < RB; ++q)
            if (q < nr) shift_rhs(base_out, r0 + q, gg.V).store(i, acc[q]);
        return;
    }
    hop_site_multi<DAG, RB>(gg, c, i, src, nr, Ug, -kappa, acc);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            Cx<T> psi[12], o[12];
            const T sp = load_s(src[q], i, psi);
            const T sc = clover_site_s(Cg, i, psi, o) * sp;
#pragma unroll
            for (int a = 0; a < 12; ++a)
                o[a] = Cx<T>{fma(sc, o[a].r, acc[q][a].r), fma(sc, o[a].i, acc[q][a].i)};
            shift_rhs(base_out, r0 + q, gg.V).store(i, o);
        }
}

template <int RB, class SP, class GA, class CL>
static int dirac_batch_run(DiracBatch<SP, GA, CL> &B, const BatchSpec &spec, bool dag, int threads, cudaStream_t s)
{
    const Geom &g0 = spec.ops[0]->gauge->lat->g;
    const bool cube = g0.lb[0] == g0.lb[1] && g0.lb[1] == g0.lb[2] && g0.lb[2] == g0.lb[3];
    B.n = spec.n;
    B.rhs_fast = spec.rhs_fast;
    int acc = 0;
    for (int k = 0; k < spec.n; ++k) {
        const Geom &g = spec.ops[k]->gauge->lat->g;
        B.g[k] = g;
        B.nrhs[k] = spec.nrhs[k];
        B.nsb[k] = grid_for(g.V, threads);
        B.ngrp[k] = (spec.nrhs[k] + RB - 1) / RB;
        acc += B.nsb[k] * B.ngrp[k];
        B.end[k] = acc;
        B.kappa[k] = (typename SP::Real)spec.ops[k]->kappa;
    }
#define MGC_DB_LAUNCH(L)                                                       \
    do {                                                                       \
        if (dag) k_dirac_batch<true, L, RB><<<acc, threads, 0, s>>>(B);        \
        else k_dirac_batch<false, L, RB><<<acc, threads, 0, s>>>(B);           \
    } while (0)
    if (cube && g0.lvb == 8) MGC_DB_LAUNCH(8);
    else if (cube && g0.lvb == 4) MGC_DB_LAUNCH(4);
    else MGC_DB_LAUNCH(0);
#undef MGC_DB_LAUNCH
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

template <class SP, class GA, class CL>
static int dirac_batch_rb(DiracBatch<SP, GA, CL> &B, const BatchSpec &spec, bool dag, int rb, int threads,
                          cudaStream_t s)
{
    if (rb == 4) return dirac_batch_run<4>(B, spec, dag, threads, s);
    if (rb == 2) return dirac_batch_run<2>(B, spec, dag, threads, s);
    return dirac_batch_run<1>(B, spec, dag, threads, s);
}

}  // namespace

// per storage precision (dirac_batch64.cu, dirac_batch32.cu, dirac_batch16.cu)
int dirac_batch_64(const BatchSpec &spec, bool dag, const void *const *in, void *const *out, int rb, int threads,
                   cudaStream_t s);
int dirac_batch_32(const BatchSpec &spec, bool dag, const void *const *in, void *const *out, int rb, int threads,
                   cudaStream_t s);
int dirac_batch_16(const BatchSpec &spec, bool dag, const void *const *in, void *const *out, int rb, int threads,
                   cudaStream_t s);

}  // namespace mgc
