// Host-side internals shared by the library's translation units: handle
// structs, error reporting and the kernel launchers each unit provides.
#pragma once

#include <cuda_runtime.h>

#include <string>

#include "mgc.h"
#include "mgc_device.cuh"

struct mgc_lattice_s {
    mgc::Geom g;
    int dims[4];
    int block[4];
};

// A gauge field keeps an FP64 copy (outer solver, force, clover build) and one
// copy at every precision from FP32 down to its storage precision: FP32 for the
// inner Krylov operator of the two-level solve, FP16 for the smoother.
struct mgc_gauge_s {
    mgc_lattice_s *lat;
    double2 *U64;  // packed FP64, 18 reals per link
    void *U32;     // packed FP32 at compress (NULL when prec == 64)
    void *U16;     // packed FP16 at compress (NULL unless prec == 16)
    int prec;      // storage precision: 64, 32 or 16
    int compress;  // 18 or 12 for the FP32/FP16 copies
};

namespace mgc {
struct SolverWork;
}

struct mgc_clover_s {
    mgc_gauge_s *gauge;
    double kappa, csw;
    double2 *C64;   // packed FP64 clover C
    double2 *Ci64;  // packed FP64 C^-1
    void *C32;      // packed FP32 C (NULL when prec == 64)
    void *C16;      // packed FP16 C followed by its per-site scales (prec == 16)
    float *C16_sc;
    void *Ci32;     // C^-1 at FP32 and FP16 (same layouts), for A = C^-1 D
    void *Ci16;
    float *Ci16_sc;
    int *d_status;  // device status word: bits set by kernels whose bounded waits ran out
    mgc::SolverWork *work;
};

namespace mgc {
// MGC_ERR_TIMEOUT if a kernel of this operator recorded a timed-out wait
// (reads and clears the device status word; synchronises the stream)
int check_device_status(const mgc_clover_s *op, cudaStream_t s);
}

// true when the operator holds a copy of its fields at precision prec
inline bool has_prec(const mgc_gauge_s *g, int prec)
{
    return prec == 64 || (prec == 32 && g->prec <= 32) || (prec == 16 && g->prec == 16);
}

namespace mgc {

int fail(int code, const std::string &msg);
int cuda_fail(cudaError_t e, const char *what, const char *file, int line);
int ok();

#define MGC_CUDA(call)                                                        \
    do {                                                                      \
        cudaError_t e_ = (call);                                              \
        if (e_ != cudaSuccess) return mgc::cuda_fail(e_, #call, __FILE__, __LINE__); \
    } while (0)

#define MGC_TRY(call)                 \
    do {                              \
        int st_ = (call);             \
        if (st_ != MGC_OK) return st_; \
    } while (0)

inline int grid_for(long long n, int threads) { return (int)((n + threads - 1) / threads); }

// Process-wide counters of kernel launches and of their algorithmic
// (compulsory) bytes: every field a launch must read or write, counted once.
void count(long long launches, double bytes);
// per-site compulsory bytes of a packed spinor, of the four forward links and
// of the clover term at each storage format
double spinor_site_bytes(int prec);
double links_site_bytes(int prec, int compress);
double clover_site_bytes(int prec);

// packed buffer sizes
size_t spinor_bytes(const Geom &g, int prec, int nrhs);
size_t gauge_bytes(const Geom &g, int prec, int compress);
size_t clover_bytes(const Geom &g, int prec);  // includes FP16 scales

// dirac.cu
int launch_pack(const Geom &g, int prec, int nrhs, const double *canon, void *packed, cudaStream_t s);
int launch_unpack(const Geom &g, int prec, int nrhs, const void *packed, double *canon, cudaStream_t s);
int launch_convert(const Geom &g, int nrhs, int pin, const void *in, int pout, void *out, cudaStream_t s);
int launch_gauge_pack(const Geom &g, const double *canon_dev, int prec, int compress, void *out, cudaStream_t s);
int launch_dirac(const mgc_clover_s *op, int prec, bool dag, const void *in, void *out, int nrhs,
                 cudaStream_t s);
// w = D z with the FP32 operator for an FP16 z (FP32 result)
int launch_dirac_from16(const mgc_clover_s *op, const void *in16, void *out32, cudaStream_t s);
int launch_clover_apply(const mgc_clover_s *op, int prec, bool inverse, const void *in, void *out, int nrhs,
                        cudaStream_t s);
int launch_gamma5(const Geom &g, int nrhs, const double2 *in, double2 *out, cudaStream_t s);
// out = A in with A = C^-1 D (QWS's clover-preconditioned operator)
int launch_apply_A(const mgc_clover_s *op, int prec, const void *in, void *out, int nrhs, cudaStream_t s);
// out (packed FP32) = s * in (packed FP64); x (packed FP64) += (cr + i ci) * e (packed FP32)
int launch_scale_to32(const Geom &g, const double2 *in, void *out, double s, cudaStream_t st);
int launch_axpy_from32(const Geom &g, double2 *x, const void *e, double cr, double ci, cudaStream_t st);

// clover_build.cu
int launch_clover_build(const Geom &g, const double2 *U64, double kappa, double csw, double2 *C64, double2 *Ci64,
                        int *d_bad, cudaStream_t s);
int launch_clover_lowprec(const Geom &g, const double2 *C64, int prec, void *out, cudaStream_t s);
int launch_clover_export(const Geom &g, const double2 *C64, double *out, cudaStream_t s);
int launch_unitarity(const Geom &g, const double *canon_dev, double *d_maxerr, cudaStream_t s);

// sap.cu
int launch_sap(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_mr,
               int x_is_zero, cudaStream_t s);
int selftest_bounded_wait(long long limit_ns, int arrive, int *flag_out, cudaStream_t s);
int fma_peak(int prec, double *flops, cudaStream_t s);
// the smoother for D with even-odd preconditioned MR domain solves
int launch_sap_eo(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_mr,
                  int x_is_zero, cudaStream_t s);
// the smoother for A = C^-1 D: n_jacobi Jacobi iterations per domain
int launch_sap_A(const mgc_clover_s *op, int prec, const void *b, void *x, int nrhs, int n_cy, int n_jacobi,
                 int x_is_zero, cudaStream_t s);

// solver.cu
int solve(mgc_clover_s *op, const double *b, double *x, int nrhs, const mgc_solve_params *p, mgc_solve_info *info,
          cudaStream_t s);
void free_work(mgc_clover_s *op);
// mgc_solve_noalloc: flexible BiCGStab with its workspace in a static device array
int solve_noalloc(mgc_clover_s *op, const double *b, double *x, const mgc_solve_params *p, mgc_solve_info *info,
                  cudaStream_t s);
// solve D x = b for one packed FP64 field already on the device (x holds the guess if guess != 0)
int solve_packed(mgc_clover_s *op, const double2 *b, double2 *x, const mgc_solve_params *p, mgc_solve_info *info,
                 cudaStream_t s);

// batches (batch.cu, with kernels in dirac.cu and sap.cu): operators of the same
// storage format and domain shape; rhs_fast orders thread blocks with the
// right-hand sides of one site block (or domain) next to each other
struct BatchSpec {
    int n;
    int rhs_fast;
    const mgc_clover_s *ops[MGC_BATCH_MAX];
    int nrhs[MGC_BATCH_MAX];
};
// D (or D^dagger) on every operator: rb right-hand sides per thread (1, 2 or 4), threads per block
int launch_dirac_batch(const BatchSpec &spec, int prec, bool dag, const void *const *in, void *const *out, int rb,
                       int threads, cudaStream_t s);
int launch_sap_batch(const BatchSpec &spec, int prec, const void *const *b, void *const *x, int n_cy, int n_mr,
                     int x_is_zero, cudaStream_t s);
// per-system site kernels of the batched two-level solve (systems operator-major;
// fields are flat batch vectors, lattice k at its offset): out32 = f_s * in64 with
// f_s = scal[s] if flag[s] else 0; x64 += g_s * e32 with g_s = scal[s] if flag[s] else 0
int launch_scale_to32_batch(const BatchSpec &spec, const size_t *off, const double2 *in, float2 *out,
                            const double *scal, const int *flag, cudaStream_t s);
int launch_axpy_from32_batch(const BatchSpec &spec, const size_t *off, double2 *x, const float2 *e,
                             const double *scal, const int *flag, cudaStream_t s);

// multigrid (mg.cu; the outer solve in solver.cu)
}  // namespace mgc
struct mgc_mg_s;
namespace mgc {
// z = the two-level preconditioner applied to v (FP64 packed; vnorm = ||v||)
int mg_precond64(mgc_mg_s *M, const mgc_mg_params *p, const double2 *v, double2 *z, double vnorm, cudaStream_t s);
mgc_clover_s *mg_operator(mgc_mg_s *M);
// flexible BiCGStab with the two-level preconditioner (canonical b, x)
int mg_solve(mgc_mg_s *M, const double *b, double *x, const mgc_solve_params *p, const mgc_mg_params *mp,
             mgc_solve_info *info, cudaStream_t s);

// force.cu
int force(mgc_clover_s *op, const double *phi, double *dSdU, const mgc_solve_params *p, mgc_solve_info *info,
          double *action, cudaStream_t s);

}  // namespace mgc
