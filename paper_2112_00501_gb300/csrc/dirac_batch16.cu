// Batched multi-RHS D with FP16 storage: the batch layout of dirac_batch.cuh
// with the FP16 operator's arithmetic (hop16.cuh), each link's stored halves
// loaded once and applied to RB right-hand sides; per right-hand side the
// operations and their order are those of the single-lattice FP16 operator,
// so results are bit-identical to it.
#include "dirac_batch.cuh"
#include "hop16.cuh"

namespace mgc {

namespace {

// acc[q] += -kappa (the two hops along MU) for RB right-hand sides sharing
// each link load
template <int MU, bool DAG, int RB, class GA>
__device__ __forceinline__ void hop16_dir_multi(const Geom &g, const int c[4], int i, const Spinor16 (&in)[RB],
                                                int nr, const GA &U, float mk, float (&ar)[RB][12],
                                                float (&ai)[RB][12])
{
    constexpr int SF = DAG ? +1 : -1;
    constexpr int SB = -SF;
    bool wr;
    uint32_t s[12], h[6], u[9];
    float wre[6], wim[6];
    int j = neighbour(g, c, MU, +1, &wr);
    bool flip = MU == 3 && wr && g.tbc < 0;
    links16(U, i, MU, u);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            words16(in[q], j, s);
            float coef = mk * in[q].scale_of(j);
            if (flip) coef = -coef;
            project16<MU, SF>(s, h);
            su3_mul16<false>(u, h, wre, wim);
            reconstruct16<MU, SF>(ar[q], ai[q], wre, wim, coef);
        }
    j = neighbour(g, c, MU, -1, &wr);
    flip = MU == 3 && wr && g.tbc < 0;
    links16(U, j, MU, u);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            words16(in[q], j, s);
            float coef = mk * in[q].scale_of(j);
            if (flip) coef = -coef;
            project16<MU, SB>(s, h);
            su3_mul16<true>(u, h, wre, wim);
            reconstruct16<MU, SB>(ar[q], ai[q], wre, wim, coef);
        }
}

template <bool DAG, int LVB, int RB, class GA>
__global__ void __launch_bounds__(256, dirac_batch_min_blocks<RB, Spinor16>())
    k_dirac16_batch(DiracBatch<Spinor16, GA, Clover16> B)
{
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
    Clover16 Cg = B.C[k];
    Spinor16 base_in = B.in[k], base_out = B.out[k];
    if (LVB > 0) {
        gg.lvb = LVB;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LVB / 4;
        base_in.lvb = base_out.lvb = Ug.lvb = Cg.lvb = LVB;
    }
    Spinor16 src[RB];
#pragma unroll
    for (int q = 0; q < RB; ++q) src[q] = shift_rhs(base_in, r0 + (q < nr ? q : 0), gg.V);
    int c[4];
    site_coords(gg, i, c);
    float ar[RB][12], ai[RB][12];
    const float csc = __ldg(Cg.sc + i);
#pragma unroll
    for (int q = 0; q < RB; ++q) {
#pragma unroll
        for (int a = 0; a < 12; ++a) ar[q][a] = ai[q][a] = 0.f;
        if (q < nr) {
            uint32_t v[12];
            words16(src[q], i, v);
            clover16_site(Cg, i, v, csc * src[q].scale_of(i), ar[q], ai[q]);
        }
    }
    const float mk = -B.kappa[k];
    hop16_dir_multi<0, DAG, RB>(gg, c, i, src, nr, Ug, mk, ar, ai);
    hop16_dir_multi<1, DAG, RB>(gg, c, i, src, nr, Ug, mk, ar, ai);
    hop16_dir_multi<2, DAG, RB>(gg, c, i, src, nr, Ug, mk, ar, ai);
    hop16_dir_multi<3, DAG, RB>(gg, c, i, src, nr, Ug, mk, ar, ai);
#pragma unroll
    for (int q = 0; q < RB; ++q)
        if (q < nr) {
            Cx<float> o[12];
#pragma unroll
            for (int a = 0; a < 12; ++a) o[a] = Cx<float>{ar[q][a], ai[q][a]};
            shift_rhs(base_out, r0 + q, gg.V).store(i, o);
        }
}

template <int RB, class GA>
static int dirac16_batch_run(DiracBatch<Spinor16, GA, Clover16> &B, const BatchSpec &spec, bool dag, int threads,
                             cudaStream_t s)
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
        B.kappa[k] = (float)spec.ops[k]->kappa;
    }
#define MGC_DB16_LAUNCH(L)                                                      \
    do {                                                                        \
        if (dag) k_dirac16_batch<true, L, RB><<<acc, threads, 0, s>>>(B);       \
        else k_dirac16_batch<false, L, RB><<<acc, threads, 0, s>>>(B);          \
    } while (0)
    if (cube && g0.lvb == 8) MGC_DB16_LAUNCH(8);
    else if (cube && g0.lvb == 4) MGC_DB16_LAUNCH(4);
    else MGC_DB16_LAUNCH(0);
#undef MGC_DB16_LAUNCH
    MGC_CUDA(cudaGetLastError());
    return MGC_OK;
}

template <class GA>
static int dirac16_batch_rb(DiracBatch<Spinor16, GA, Clover16> &B, const BatchSpec &spec, bool dag, int rb,
                            int threads, cudaStream_t s)
{
    if (rb == 4) return dirac16_batch_run<4>(B, spec, dag, threads, s);
    if (rb == 2) return dirac16_batch_run<2>(B, spec, dag, threads, s);
    return dirac16_batch_run<1>(B, spec, dag, threads, s);
}

}  // namespace

int dirac_batch_16(const BatchSpec &spec, bool dag, const void *const *in, void *const *out, int rb, int threads,
                   cudaStream_t s)
{
    const mgc_gauge_s *ga0 = spec.ops[0]->gauge;
    if (ga0->compress == 12) {
        DiracBatch<Spinor16, Gauge16x12, Clover16> B;
        for (int k = 0; k < spec.n; ++k) {
            const mgc_clover_s *op = spec.ops[k];
            const Geom &g = op->gauge->lat->g;
            B.in[k] = sp16(g, in[k], spec.nrhs[k]);
            B.out[k] = sp16(g, out[k], spec.nrhs[k]);
            B.U[k] = Gauge16x12{(uint2 *)op->gauge->U16, g.lvb};
            B.C[k] = cl16(g, op);
        }
        return dirac16_batch_rb(B, spec, dag, rb, threads, s);
    } else {
        DiracBatch<Spinor16, Gauge16x18, Clover16> B;
        for (int k = 0; k < spec.n; ++k) {
            const mgc_clover_s *op = spec.ops[k];
            const Geom &g = op->gauge->lat->g;
            B.in[k] = sp16(g, in[k], spec.nrhs[k]);
            B.out[k] = sp16(g, out[k], spec.nrhs[k]);
            B.U[k] = Gauge16x18{(uint32_t *)op->gauge->U16, g.lvb};
            B.C[k] = cl16(g, op);
        }
        return dirac16_batch_rb(B, spec, dag, rb, threads, s);
    }
}

}  // namespace mgc
