// Batched multi-RHS D with FP64 storage (kernel in dirac_batch.cuh).
#include "dirac_batch.cuh"

namespace mgc {

int dirac_batch_64(const BatchSpec &spec, bool dag, const void *const *in, void *const *out, int rb, int threads,
                   cudaStream_t s)
{
    DiracBatch<Spinor64, Gauge64, Clover64> B;
    for (int k = 0; k < spec.n; ++k) {
        const mgc_clover_s *op = spec.ops[k];
        const Geom &g = op->gauge->lat->g;
        B.in[k] = sp64(g, in[k]);
        B.out[k] = sp64(g, out[k]);
        B.U[k] = Gauge64{op->gauge->U64, g.lvb};
        B.C[k] = Clover64{op->C64, g.lvb};
    }
    return dirac_batch_rb(B, spec, dag, rb, threads, s);
}

}  // namespace mgc
