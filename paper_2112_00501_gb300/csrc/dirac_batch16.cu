// Batched multi-RHS D with FP16 storage (kernel in dirac_batch.cuh).
#include "dirac_batch.cuh"

namespace mgc {

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
        return dirac_batch_rb(B, spec, dag, rb, threads, s);
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
        return dirac_batch_rb(B, spec, dag, rb, threads, s);
    }
}

}  // namespace mgc
