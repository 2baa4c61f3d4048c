// Batched multi-RHS D with FP32 storage (kernel in dirac_batch.cuh).
#include "dirac_batch.cuh"

namespace mgc {

int dirac_batch_32(const BatchSpec &spec, bool dag, const void *const *in, void *const *out, int rb, int threads,
                   cudaStream_t s)
{
    const mgc_gauge_s *ga0 = spec.ops[0]->gauge;
    if (ga0->compress == 12) {
        DiracBatch<Spinor32, Gauge32x12, Clover32> B;
        for (int k = 0; k < spec.n; ++k) {
            const mgc_clover_s *op = spec.ops[k];
            const Geom &g = op->gauge->lat->g;
            B.in[k] = sp32(g, in[k]);
            B.out[k] = sp32(g, out[k]);
            B.U[k] = Gauge32x12{(float4 *)op->gauge->U32, g.lvb};
            B.C[k] = Clover32{(float4 *)op->C32, g.lvb};
        }
        return dirac_batch_rb(B, spec, dag, rb, threads, s);
    } else {
        DiracBatch<Spinor32, Gauge32x18, Clover32> B;
        for (int k = 0; k < spec.n; ++k) {
            const mgc_clover_s *op = spec.ops[k];
            const Geom &g = op->gauge->lat->g;
            B.in[k] = sp32(g, in[k]);
            B.out[k] = sp32(g, out[k]);
            B.U[k] = Gauge32x18{(float2 *)op->gauge->U32, g.lvb};
            B.C[k] = Clover32{(float4 *)op->C32, g.lvb};
        }
        return dirac_batch_rb(B, spec, dag, rb, threads, s);
    }
}

}  // namespace mgc
