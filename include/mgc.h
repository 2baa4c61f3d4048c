/*
 * mgc.h -- C ABI of the GB300 clover-Wilson Dirac operator, SAP smoother,
 * flexible outer solver and link force (arXiv:2112.00501, "Multigrid Solver on
 * Fugaku": the fine-grid operator of Eq. (1) and the QWS smoother M_SAP of
 * Sec. 2 used as the post-smoother of Sec. 3).
 *
 * Conventions (the paper fixes none of them; these are the library's readings):
 *   D = C - kappa*H,  H psi(x) = sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                                       + (1 + gamma_mu) U_mu(x-mu)^+ psi(x-mu)],
 *   C = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}   (Eq. (1)),
 *   F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^+)/8 (four-leaf clover, no trace
 *   subtraction), chiral gamma basis with gamma_5 = diag(1, 1, -1, -1), so C is
 *   two 6x6 Hermitian blocks; periodic in x, y, z and periodic (t_bc = +1) or
 *   antiperiodic (t_bc = -1) in t, applied to the hops that cross t = Lt-1 <-> 0.
 *
 * Canonical external layouts (complex128 = two doubles, real then imaginary):
 *   site  s = x + Lx*(y + Ly*(z + Lz*t))
 *   spinor  [nrhs][s][spin 4][colour 3]       (24 doubles per site)
 *   gauge   [s][mu 4][row 3][col 3]           (U_mu(s) links s to s+mu)
 *   clover  [s][12][12], index spin*3+colour  (export only)
 *   force   [s][mu 4][row 3][col 3]           (dS/dRe U + i dS/dIm U)
 *
 * Packed device layouts ("packed spinors") are what the operator, smoother and
 * conversion calls take.  Sites are ordered block by block (the SAP domains of
 * the lattice), and inside a block even sites come before odd sites; each
 * precision stores a site's 24 reals as planes of 16-byte vectors so that
 * consecutive sites are consecutive in memory:
 *   prec 64: 12 planes of double2 per block, [rhs][block][plane][site]
 *   prec 32:  6 planes of float4
 *   prec 16:  3 planes of 8 halves, then (after all rhs' planes) one float
 *             scale per site; the stored halves are value/scale and the scale
 *             is the site's largest |real component|.
 * mgc_spinor_bytes() gives the size; mgc_spinor_pack()/unpack() convert.
 *
 * Ownership: the caller owns every buffer it passes (for example a torch
 * tensor's data pointer); the library never frees them.  Handles own the
 * library's packed copies of the gauge field and clover term and any solver
 * workspace, and release them in the matching destroy call.
 *
 * Streams: `stream` is a cudaStream_t passed as void* (NULL = legacy default
 * stream).  Operator, smoother and conversion calls only enqueue work on it.
 * mgc_solve and mgc_force synchronise the stream (they read convergence
 * scalars back to the host).
 *
 * Errors: every call returns an MGC_* status; mgc_status_string() names it and
 * mgc_last_error() returns a message for the last failing call of the calling
 * host thread.  No call aborts the process.
 */
#ifndef MGC_H
#define MGC_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define MGC_OK 0
#define MGC_ERR_INVALID_ARG 1       /* NULL handle/pointer, bad enum value */
#define MGC_ERR_UNSUPPORTED_SHAPE 2 /* dims not divisible by block, odd block count, ... */
#define MGC_ERR_NOT_UNITARY 3       /* 12-real compression asked for a non-SU(3) field */
#define MGC_ERR_CUDA 4              /* a CUDA runtime call failed (see mgc_last_error) */
#define MGC_NOT_CONVERGED 5         /* solver hit max_iter; info holds the residual */
#define MGC_ERR_BREAKDOWN 6         /* NaN/Inf or a zero denominator in the solver */
#define MGC_ERR_TIMEOUT 7           /* a bounded device wait ran out */
#define MGC_ERR_NO_DEVICE 8         /* no usable sm_103 device */

/* storage precisions */
#define MGC_PREC_64 64
#define MGC_PREC_32 32
#define MGC_PREC_16 16

typedef struct mgc_lattice_s *mgc_lattice_t;
typedef struct mgc_gauge_s *mgc_gauge_t;
typedef struct mgc_clover_s *mgc_clover_t;

const char *mgc_status_string(int status);
const char *mgc_last_error(void);
int mgc_version(void);

/*
 * Process-wide counters kept by the library (no paper counterpart; they make
 * throughput measurable): the number of this library's kernel launches and
 * the algorithmic bytes of those launches, i.e. every field a launch must
 * read or write counted once (spinors, links, clover, Krylov vectors at
 * their storage precision).  reset != 0 zeroes both after reading.
 */
int mgc_counters(long long *launches, double *algorithmic_bytes, int reset);

/*
 * Lattice geometry with SAP domains (Sec. 2: the domain-decomposed smoother).
 * dims = (Lx, Ly, Lz, Lt); block = SAP domain extents, each a power of two >= 2
 * with dims[mu] / block[mu] even (so the red/black colouring of domains is
 * consistent across the periodic wrap) and at most 1024 sites per domain.
 * t_bc = +1 (periodic) or -1 (antiperiodic) in t.
 * Errors: INVALID_ARG for a NULL out or bad t_bc, UNSUPPORTED_SHAPE otherwise.
 */
int mgc_lattice_create(const int dims[4], const int block[4], int t_bc, mgc_lattice_t *out);
int mgc_lattice_destroy(mgc_lattice_t lat);
long long mgc_lattice_volume(mgc_lattice_t lat);

/* Bytes of a packed spinor buffer holding nrhs fields at precision prec. */
size_t mgc_spinor_bytes(mgc_lattice_t lat, int prec, int nrhs);

/*
 * Canonical complex128 spinors (device pointer, nrhs fields) to the packed
 * layout at precision prec, and back.  Rounding to FP32/FP16 is to nearest
 * even; prec 16 stores a per-site scale.  Asynchronous on stream.
 */
int mgc_spinor_pack(mgc_lattice_t lat, int prec, int nrhs, const double *canonical, void *packed,
                    void *stream);
int mgc_spinor_unpack(mgc_lattice_t lat, int prec, int nrhs, const void *packed, double *canonical,
                      void *stream);
/* packed precision conversion (same lattice, same nrhs) */
int mgc_spinor_convert(mgc_lattice_t lat, int nrhs, int prec_in, const void *in, int prec_out,
                       void *out, void *stream);

/*
 * Gauge field U (canonical complex128, V*4*9 entries; host memory if
 * on_device == 0, else device memory).  The handle keeps an FP64 copy for the
 * outer solver, an FP32 copy when storage_prec <= 32 (inner Krylov operator)
 * and an FP16 copy when storage_prec == 16 (smoother); the low-precision
 * copies use compress = 18 (full matrices) or 12 (rows 0 and 1; row 2 is rebuilt as
 * conj(row0 x row1), which needs SU(3) links: with compress = 12 the call
 * returns MGC_ERR_NOT_UNITARY when any link's unitarity or determinant error
 * exceeds 1e-10).  Synchronises stream.
 */
int mgc_gauge_create(mgc_lattice_t lat, const double *U, int on_device, int storage_prec,
                     int compress, void *stream, mgc_gauge_t *out);
int mgc_gauge_destroy(mgc_gauge_t g);

/*
 * The clover-Wilson operator D = C - kappa*H (Eq. (1)).  C and C^-1 are
 * computed on the GPU in FP64 from the gauge field's clover leaves (Sec. 2:
 * computing C and C^-1 from the gauge field); copies of C at FP32 and FP16
 * follow the gauge field's copies.  The gauge handle must outlive
 * the operator.  Synchronises stream.
 */
int mgc_clover_create(mgc_gauge_t g, double kappa, double csw, void *stream, mgc_clover_t *out);
int mgc_clover_destroy(mgc_clover_t op);
/*
 * The operator's device status word (no paper counterpart): kernels that wait
 * on their own asynchronous copies give up after a bounded time and set a bit
 * here instead of hanging.  *flags receives the word; clear != 0 zeroes it.
 * Returns MGC_ERR_TIMEOUT when any bit is set.  Synchronises stream.
 * mgc_solve and mgc_force check it themselves.  After MGC_ERR_TIMEOUT the
 * results of the calls since the last check are invalid and the operator
 * must be destroyed, not reused: a copy that never completed may still land
 * in memory the next launch uses.
 */
int mgc_device_status(mgc_clover_t op, int *flags, int clear, void *stream);
/*
 * Self-test of that bounded-wait mechanism (no paper counterpart): one thread
 * block waits on a shared-memory barrier for at most limit_ns (<= 2 s).  With
 * arrive != 0 the barrier completes and the call returns MGC_OK; with
 * arrive == 0 nothing arrives, the wait runs out, *flag_out is non-zero and the
 * call returns MGC_ERR_TIMEOUT with the context still usable.
 */
int mgc_selftest_bounded_wait(long long limit_ns, int arrive, int *flag_out, void *stream);
/*
 * Measured fused multiply-add rate of this GPU (no paper counterpart; the
 * denominator of the roofline of the arithmetic-bound kernels): prec 32 (FP32
 * FMA) or 64 (FP64 FMA).  Eight 256-thread blocks per SM, each thread running
 * eight independent FMA chains; *flops_per_s receives 2 x FMAs / time of the
 * fastest of five launches (about 10 ms each).  Synchronises stream.
 */
int mgc_fma_peak(int prec, double *flops_per_s, void *stream);
/* C (inverse = 0) or C^-1 (inverse = 1) as canonical 12x12 complex128 per site (device). */
int mgc_clover_export(mgc_clover_t op, int inverse, double *out, void *stream);

/*
 * out = D in and out = D^dagger in (= gamma5 D gamma5 in) for nrhs packed
 * spinors at precision prec (64, or 32/16 when the gauge keeps that copy).  Eq. (1).
 * in and out must not overlap.  Asynchronous on stream.
 */
int mgc_apply_D(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, void *stream);
int mgc_apply_Ddag(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, void *stream);

/*
 * out = C in (inverse = 0) or C^-1 in (inverse = 1), site-local two 6x6
 * Hermitian blocks (Eq. (1); C^-1 is what QWS applies before M_SAP, Sec. 3),
 * at any precision the operator keeps.
 */
int mgc_apply_clover(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, int inverse,
                     void *stream);

/*
 * Multiplicative SAP (Sec. 2, M_SAP; Sec. 3, post-smoother): n_cy sweeps, each
 * visiting the red domains then the black domains; for every domain B,
 * x_B += MR_{n_mr}(D_B, (b - D x)|_B) with D_B the Dirichlet domain operator
 * and n_mr minimal-residual steps from zero.  x (packed, prec) is updated in
 * place; x_is_zero = 1 promises x == 0 on entry and skips its first residual.
 * prec 64 computes in FP64; 32 and 16 compute in FP32, where a domain whose
 * <p, p> falls below FP32's normal range takes no further MR step (alpha = 0)
 * and an FP16-stored site below that range is stored as zero.  Asynchronous.
 */
int mgc_sap_smooth(mgc_clover_t op, const void *b, void *x, int nrhs, int n_cy, int n_mr,
                   int prec, int x_is_zero, void *stream);

/*
 * mgc_sap_smooth with the even-odd preconditioned MR domain solver of
 * DD-alphaAMG (which the paper's multigrid follows, Sec. 3): on each domain,
 * n_mr MR steps on the even-site Schur complement
 * C_ee - kappa^2 H_eo C_oo^-1 H_oe with source r_e + kappa H_eo C_oo^-1 r_o, then
 * e_o = C_oo^-1 (r_o + kappa H_oe e_e).  Same arguments as mgc_sap_smooth.
 */
int mgc_sap_smooth_eo(mgc_clover_t op, const void *b, void *x, int nrhs, int n_cy, int n_mr, int prec,
                      int x_is_zero, void *stream);

/*
 * QWS's clover-preconditioned operator (Sec. 2): out = A in with
 * A = C^-1 D = 1 - kappa C^-1 H, for nrhs packed spinors at precision prec
 * (64, or 32/16 when the gauge keeps that copy).  Asynchronous.
 */
int mgc_apply_A(mgc_clover_t op, const void *in, void *out, int nrhs, int prec, void *stream);

/*
 * QWS's M_SAP for A (Sec. 2): n_cy multiplicative sweeps (red domains, then
 * black) on A x = b, each domain B getting x_B += e with e from n_jacobi
 * Jacobi iterations e <- r_B + kappa C_B^-1 H_B e on the Dirichlet domain
 * operator A_B from e = 0, r_B = (b - A x)|_B.  x (packed, prec) is updated in
 * place; x_is_zero = 1 promises x == 0 on entry.  prec 64 computes in FP64;
 * 32 and 16 compute in FP32.  Asynchronous.
 */
int mgc_sap_smooth_A(mgc_clover_t op, const void *b, void *x, int nrhs, int n_cy, int n_jacobi, int prec,
                     int x_is_zero, void *stream);

/*
 * Solver parameters (Sec. 3: flexible outer solver with the SAP smoother as
 * preconditioner; Sec. 2: QWS's double-precision Richardson iteration around a
 * single-precision solver).  Methods:
 *   0  FGCR(restart) with FP64 Krylov vectors, FP64 D in every iteration;
 *   1  flexible BiCGStab (the paper's outer solver) with FP64 vectors;
 *   2  two-level: FP64 defect correction (residual b - D x, D, x and the
 *      residual norm in FP64) around an FP32 FGCR(restart) + SAP inner solve
 *      to inner_tol: FP32 Krylov vectors and orthogonalisation, inner
 *      products summed in FP32 over a few entries per thread and in FP64
 *      across the lattice, FP64 Gram-Schmidt coefficients;
 *   3  QWS (Sec. 2): FP64 Richardson on b - D x around an FP32 BiCGStab on
 *      A M_SAP (A = C^-1 D, source C^-1 r, M_SAP from mgc_sap_smooth_A with
 *      n_mr Jacobi iterations per domain) to inner_tol; x += ||C^-1 r|| M_SAP y.
 */
typedef struct {
    int method;        /* 0, 1, 2 or 3 (above) */
    int precond;       /* 0 = none, 1 = SAP */
    int smoother_prec; /* 64, 32 or 16 (needs a copy at that precision; 32/16 for method 2) */
    int n_cy;          /* SAP sweeps per preconditioner application */
    int n_mr;          /* MR steps per domain */
    int restart;       /* FGCR length m (<= 32); method 2: inner iterations per pass */
    double tol;        /* stop when ||b - D x|| <= tol ||b||, D in FP64 */
    int max_iter;      /* preconditioner applications (methods 0, 2), BiCGStab iterations (1, 3) */
    int on_device;     /* 1: b, x are device pointers; 0: host pointers */
    int x_is_guess;    /* 1: x holds the initial guess; 0: start from x = 0 */
    double inner_tol;  /* method 2: relative residual reduction of each inner solve */
    int sap_solver;    /* SAP domain solver of methods 0-2: 0 = MR, 2 = even-odd preconditioned MR */
} mgc_solve_params;

typedef struct {
    int status;        /* MGC_OK, MGC_NOT_CONVERGED or MGC_ERR_BREAKDOWN */
    int iters;         /* preconditioned iterations (max over right-hand sides) */
    int restarts;      /* true-residual recomputations (method 2: outer passes) */
    double true_res;   /* max over rhs of ||b - D x|| / ||b|| in FP64 */
} mgc_solve_info;

void mgc_solve_params_default(mgc_solve_params *p);

/*
 * Solve D x = b for nrhs canonical complex128 right-hand sides (one after the
 * other) with the method of p (above): methods 0, 1 and the outer iteration
 * of 3 keep their vectors, inner products, orthogonalisation and residual
 * updates in FP64; method 2 keeps its residual, x and norms in FP64 and runs
 * its inner solve in FP32 (above); the SAP preconditioner in smoother_prec.
 * The solve is scale invariant for every source whose squared norm is a
 * normal FP64 number: method 2 hands its inner solve each outer residual
 * multiplied by a power of two that brings its rms near 1, methods 0 and 1
 * solve D (u x) = u b for a source whose rms lies beyond 2^+-30 (u a power
 * of two), method 3 normalises its inner source.
 * Synchronises stream.
 * Host pointers (on_device = 0): with x in page-locked memory, method 2
 * copies x back on a stream of its own while the FP64 residual that confirms
 * convergence is computed; x holds the solution once the call returns, as
 * with pageable x, and is not written after the return.  With several
 * right-hand sides in page-locked b, the next b is copied to the device
 * while the current one is solved (in a second 24 * 8 * V byte buffer of the
 * operator's workspace); b is not read after the return.
 */
int mgc_solve(mgc_clover_t op, const double *b, double *x, int nrhs, const mgc_solve_params *p,
              mgc_solve_info *info, void *stream);

/*
 * mgc_solve without any allocation.  The paper has no counterpart: this entry
 * point is for callers that cannot call cudaMalloc at solve time -- for example
 * code whose device memory is all owned by another allocator (a framework's
 * caching pool or a fixed memory budget), or a loop that cannot afford the
 * device-wide synchronisation a cudaMalloc/cudaFree pair brings.  It solves
 * D x = b for one right-hand side with flexible BiCGStab (p->method must be 1)
 * and performs no cudaMalloc, cudaFree or other allocation: its workspace is a
 * file-scope device array of fixed size (about 10.5 MB, held by every GPU that
 * loads the library until the process exits), which limits the lattice to
 * MGC_NOALLOC_MAX_SITES sites; larger lattices return
 * MGC_ERR_UNSUPPORTED_SHAPE.  b and x are canonical complex128 device pointers
 * (p->on_device must be 1); the operator handle (created beforehand) supplies
 * D and the smoother.
 * The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress), so make that first call before any stream capture.
 * The address is cached per device for the life of the process; after
 * cudaDeviceReset (or any other teardown of the device's primary context) the
 * cached address is stale and this entry point must not be called again.
 * All calls share the one array and it keeps the last call's contents; calls
 * that overlap on the GPU (other streams, other host threads) race on it and
 * must not be made: serialise calls from several host threads.  Synchronises
 * stream.
 */
#define MGC_NOALLOC_MAX_SITES 4096
int mgc_solve_noalloc(mgc_clover_t op, const double *b, double *x, const mgc_solve_params *p, mgc_solve_info *info,
                      void *stream);

/*
 * Link force of S = phi^+ (D^+ D)^-1 phi: solves D^+ Y = phi (as
 * gamma5 D^-1 gamma5 phi) and D X = Y, then dS/dU from the hopping outer
 * products and the clover-leaf derivative.  phi: canonical complex128 (one
 * field, on_device as in p); dSdU: canonical [V][4][3][3] complex128 in the
 * same memory kind.  action (optional, room for two doubles) receives S,
 * estimated as 2 Re(phi^+ X) - ||D X||^2 (second order in the solver error),
 * as the unevaluated sum action[0] + action[1]: action[0] is S rounded to
 * double and action[1] the remainder, from exact products and double-double
 * sums, so that the difference of two nearby actions keeps its digits (finite
 * differences at small steps).  Synchronises stream.
 */
int mgc_force(mgc_clover_t op, const double *phi, double *dSdU, const mgc_solve_params *p,
              mgc_solve_info *info, double *action, void *stream);

/*
 * Two-level multigrid (Sec. 3), single precision inside the preconditioner.
 * Aggregates are agg[0] x agg[1] x agg[2] x agg[3] fine sites (each extent a
 * multiple of the SAP domain extent and dividing the lattice), split by
 * chirality (spins 0, 1 and spins 2, 3), so a coarse site carries 2 nvec
 * degrees of freedom (1 <= nvec <= MGC_MG_MAX_NVEC).  The prolongation P is the
 * nvec null vectors orthonormalised per aggregate and chirality (modified
 * Gram-Schmidt in vector order), the restriction is R = P^dagger and the
 * coarse operator D_c = R D P, stored as a 9-point stencil (the coupling inside
 * an aggregate and the fine hops across each of its 8 faces).  The
 * preconditioner applied to v is the coarse correction x = P D_c^-1 R v
 * (D_c^-1 by BiCGStab to coarse_tol or coarse_maxit iterations) followed by
 * n_cy sweeps of QWS's SAP for A on C^-1 (v - D x) (post-smoothing), all in
 * FP32 arithmetic.  The handle needs an operator with an FP32 copy; it does not
 * own the operator (destroy it first).
 *
 * Canonical coarse vectors are complex128 [Vc][chirality 2][nvec] with the
 * coarse sites lexicographic (x fastest) on the lattice dims / agg; the coarse
 * stencil export is complex128 [Vc][9][2 nvec][2 nvec] (row, column) with the
 * stencil order: inside, +x, -x, +y, -y, +z, -z, +t, -t, entry k applied to
 * the coarse neighbour in that direction.
 */
#define MGC_MG_MAX_NVEC 32
typedef struct mgc_mg_s *mgc_mg_t;
typedef struct {
    int n_cy;          /* post-smoother sweeps */
    int n_jacobi;      /* Jacobi iterations per domain in the post-smoother */
    int smoother_prec; /* 32 or 16 */
    double coarse_tol; /* relative residual of the coarse BiCGStab */
    int coarse_maxit;
    int n_adapt;       /* adaptive setup passes */
} mgc_mg_params;
void mgc_mg_params_default(mgc_mg_params *p);
int mgc_mg_create(mgc_clover_t op, const int agg[4], int nvec, mgc_mg_t *out);
int mgc_mg_destroy(mgc_mg_t mg);
/* coarse lattice volume */
long long mgc_mg_coarse_volume(mgc_mg_t mg);
/*
 * Setup (Sec. 3): null vectors V_i = M_SAP(C^-1 eta_i) from the nvec random
 * fields eta (canonical complex128 [nvec][V][4][3], device; the caller draws
 * them), then W and D_c; then n_adapt passes that replace every V_i by the
 * preconditioner applied to it (scaled to unit norm) and rebuild W and D_c.
 * Synchronises stream.
 */
int mgc_mg_setup(mgc_mg_t mg, const double *eta, const mgc_mg_params *p, void *stream);
/* W and D_c from given vectors V (canonical, device) without any smoothing */
int mgc_mg_set_vectors(mgc_mg_t mg, const double *V, void *stream);
/* W (canonical [nvec][V][4][3]) and D_c (layout above), both complex128 on the device */
int mgc_mg_export(mgc_mg_t mg, double *W, double *Dc, void *stream);
/* u = R v, v = P u, out = D_c u, all canonical complex128 on the device, computed in FP32 */
int mgc_mg_restrict(mgc_mg_t mg, const double *v, double *u, void *stream);
int mgc_mg_prolong(mgc_mg_t mg, const double *u, double *v, void *stream);
int mgc_mg_coarse_apply(mgc_mg_t mg, const double *u, double *out, void *stream);
/* D_c x = b by BiCGStab to tol (relative) or maxit iterations; *iters receives the count.  Synchronises. */
int mgc_mg_coarse_solve(mgc_mg_t mg, const double *b, double *x, double tol, int maxit, int *iters, void *stream);
/* x = the two-level preconditioner applied to v (canonical fine fields, device).  Synchronises. */
int mgc_mg_precond(mgc_mg_t mg, const double *v, double *x, const mgc_mg_params *p, void *stream);
/*
 * The multigrid solve (Sec. 3): flexible BiCGStab with FP64 vectors and the
 * FP64 operator, preconditioned by the two-level preconditioner, to the true
 * residual tol.  b, x canonical complex128 (one field; p->on_device as in
 * mgc_solve; p->tol and p->max_iter are used).  Synchronises.
 */
int mgc_mg_solve(mgc_mg_t mg, const double *b, double *x, const mgc_solve_params *p, const mgc_mg_params *mp,
                 mgc_solve_info *info, void *stream);

/*
 * Batches of lattices (no paper counterpart; the paper's multiple
 * right-hand sides, Sec. 4, extended to several lattices at once).  A batch
 * groups up to MGC_BATCH_MAX operators that share storage precision, link
 * compression and SAP domain shape; operator k carries nrhs[k] >= 1
 * right-hand sides.  One kernel launch then covers every lattice and every
 * right-hand side: the batched D applies one launch per call, the batched
 * smoother one launch per colour and sweep, replayed from a CUDA graph
 * captured on first use.  An autotuner times the launch shapes (right-hand
 * sides per thread, threads per block, order of the thread blocks) on first
 * use at each precision and keeps the fastest.  The batch does not own the
 * operators: destroy it before them.
 *
 * Fields passed to the batch functions are arrays of n pointers, one per
 * operator, each to nrhs[k] packed (apply, smoother) or canonical (solve)
 * fields back to back.
 */
#define MGC_BATCH_MAX 8
typedef struct mgc_batch_s *mgc_batch_t;
int mgc_batch_create(const mgc_clover_t *ops, const int *nrhs, int n, mgc_batch_t *out);
int mgc_batch_destroy(mgc_batch_t b);
/* total right-hand sides (systems) of the batch */
int mgc_batch_systems(mgc_batch_t b);
/* out_k = D in_k (dagger = 0) or D^dagger in_k for every operator k; prec as in mgc_apply_D */
int mgc_batch_apply_D(mgc_batch_t b, const void *const *in, void *const *out, int prec, int dagger, void *stream);
/*
 * mgc_sap_smooth on every operator of the batch (prec 32 or 16).  The 2 n_cy
 * launches are captured once into a CUDA graph per distinct argument set
 * (pointers, n_cy, n_mr, prec, x_is_zero; the last few are kept) and replayed.
 */
int mgc_batch_sap_smooth(mgc_batch_t b, const void *const *rhs, void *const *x, int n_cy, int n_mr, int prec,
                         int x_is_zero, void *stream);
/*
 * Solve D_k x = b for every right-hand side of every operator with the
 * two-level method (p->method must be 2, p->precond 1): FP64 defect
 * correction around an FP32 FGCR + SAP inner solve, all systems advancing in
 * lock step so that each step is one launch over the whole batch.  Every
 * system has its own Krylov coefficients, computed on the device; a system
 * that has converged stops changing.  b, x: arrays of n canonical complex128
 * pointers (nrhs[k] fields each; on_device as in p).  info: one entry per
 * system, operator-major.  Returns the worst status.  Synchronises stream.
 */
int mgc_batch_solve(mgc_batch_t b, const double *const *rhs, double *const *x, const mgc_solve_params *p,
                    mgc_solve_info *info, void *stream);
/*
 * Launch shape chosen for D at precision prec (tuning now if not yet done;
 * force != 0 re-tunes): right-hand sides per thread, threads per block and
 * whether thread blocks of one site block and different right-hand sides are
 * adjacent; and for the smoother the same block order flag.
 */
int mgc_batch_tune(mgc_batch_t b, int prec, int force, int *rhs_per_thread, int *threads, int *rhs_fast_d,
                   int *rhs_fast_sap, void *stream);
/*
 * Pin the launch shape at precision prec instead of tuning: rhs_per_thread
 * 1, 2 or 4; threads 128 or 256; rhs_fast_d, rhs_fast_sap 0 or 1.
 */
int mgc_batch_set_shape(mgc_batch_t b, int prec, int rhs_per_thread, int threads, int rhs_fast_d,
                        int rhs_fast_sap);

#ifdef __cplusplus
}
#endif

#endif /* MGC_H */
