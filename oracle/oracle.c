/*
 * oracle.c -- plain, slow FP64 CPU oracle for the clover-Wilson operator,
 * the multiplicative Schwarz alternating procedure (SAP) with block
 * minimal-residual solves, the flexible outer solvers and the gauge-link
 * force of S = phi^dagger (D^dagger D)^-1 phi.
 *
 * TEST INFRASTRUCTURE ONLY.  Only the tests, the smoke check and the
 * benchmark's CPU-baseline leg load this file's library.  The CUDA library
 * shares no code, header, table or helper with it.
 *
 * Everything here is written site by site from the definitions, with no
 * blocking, fusion or reordering:
 *   - Eq. (1): D = C + kappa*H_paper with C = 1 + (i/2) kappa c_SW
 *     sigma_{mu nu} F_{mu nu}.  The reading used here writes the hopping term
 *     with the opposite sign, D = C - kappa*H with
 *       H psi(x) = sum_mu [(1 - gamma_mu) U_mu(x) psi(x+mu)
 *                         + (1 + gamma_mu) U_mu(x-mu)^dagger psi(x-mu)],
 *     which is the standard Wilson (r = 1) operator in the kappa
 *     normalisation.
 *   - Gamma matrices in the chiral basis:
 *       gamma_k = [[0, -i sigma_k], [i sigma_k, 0]]  (k = x, y, z),
 *       gamma_t = [[0, -1], [-1, 0]],  gamma_5 = gamma_t gamma_x gamma_y gamma_z
 *     = diag(1, 1, -1, -1); sigma_{mu nu} = (i/2) [gamma_mu, gamma_nu].
 *   - F_{mu nu} = (Q_{mu nu} - Q_{mu nu}^dagger) / 8 with Q the sum of the four
 *     plaquette leaves in the mu-nu plane that start and end at x; no trace
 *     subtraction.  Summing Eq. (1) over both orders of (mu, nu) gives
 *     C = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}.
 *   - Boundary conditions: periodic in x, y, z; antiperiodic in t, applied as
 *     a factor tbc = -1 on the hopping terms that cross t = Lt-1 <-> 0.  Clover
 *     leaves use the raw links.
 *   - Sec. 2: M_SAP is a multiplicative, domain-decomposed preconditioner
 *     whose domains are visited alternately.  Here: domains are blocks of
 *     Bx*By*Bz*Bt sites coloured by the parity of their block coordinates;
 *     colour 0 (red) first, then colour 1 (black).  For each block of the
 *     current colour: r_B = (b - D x) restricted to B, e = MR_k(D_B, r_B),
 *     x_B += e, where D_B is D with every hop that leaves B dropped
 *     (Dirichlet).  MR starts at e = 0 and takes exactly k steps
 *     p = D_B r, alpha = <p, r> / <p, p>, e += alpha r, r -= alpha p.
 *   - Sec. 2, QWS: the clover-preconditioned operator A = C^-1 D, its SAP
 *     with a fixed number of Jacobi iterations per block, and the QWS solver
 *     (Richardson around BiCGStab on A M_SAP, source multiplied by C^-1).
 *   - Sec. 3, multigrid: aggregates split by chirality, block-orthonormal
 *     null vectors as prolongation, R = P^dagger, D_c = R D P as a 9-point
 *     coarse stencil, coarse BiCGStab, the two-level preconditioner (coarse
 *     correction, then SAP post-smoothing), its setup from random vectors, and
 *     the flexible-BiCGStab multigrid solve.
 *   - Sec. 3: the outer solver is flexible (the paper's is flexible BiCGStab);
 *     FGCR with restarts and flexible BiCGStab are provided, both right
 *     preconditioned with n_cy SAP sweeps from x = 0.
 *   - Force: S = ||Y||^2 with Y = D^-dagger phi and X = D^-1 Y; for a link
 *     variation, delta S = -2 Re Y^dagger (delta D) X; the returned tensor is
 *     dS/dRe U + i dS/dIm U for each link entry.
 *
 * Canonical layouts (complex double):
 *   site s = x + Lx*(y + Ly*(z + Lz*t)); spinor psi[s][spin 4][colour 3];
 *   gauge U[s][mu 4][row 3][col 3]; clover C[s][12][12] with index
 *   spin*3 + colour.
 */
#include <complex.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>
#ifdef _OPENMP
#include <omp.h>
#endif

typedef double complex cplx;

/* ------------------------------------------------------------------ */
/* lattice geometry                                                     */
/* ------------------------------------------------------------------ */

static long vol4(const int *L) { return (long)L[0] * L[1] * L[2] * L[3]; }

static void site_coords(long s, const int *L, int c[4])
{
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = (int)(s % L[mu]);
        s /= L[mu];
    }
}

static long site_index(const int c[4], const int *L)
{
    return c[0] + (long)L[0] * (c[1] + (long)L[1] * (c[2] + (long)L[2] * c[3]));
}

/* site s displaced by d[mu] in every direction, with periodic wrap */
static long shifted(long s, const int *L, const int d[4])
{
    int c[4];
    site_coords(s, L, c);
    for (int mu = 0; mu < 4; ++mu)
        c[mu] = ((c[mu] + d[mu]) % L[mu] + L[mu]) % L[mu];
    return site_index(c, L);
}

/* nearest neighbour s +- mu; *crossed = 1 if the hop wraps around the lattice */
static long neighbour(long s, int mu, int dir, const int *L, int *crossed)
{
    int c[4];
    site_coords(s, L, c);
    int v = c[mu] + dir;
    *crossed = (v < 0 || v >= L[mu]);
    c[mu] = (v + L[mu]) % L[mu];
    return site_index(c, L);
}

/* ------------------------------------------------------------------ */
/* gamma matrices, chiral basis                                         */
/* ------------------------------------------------------------------ */

static cplx G[4][4][4];         /* G[mu][row][col], mu = x, y, z, t */
static cplx G5[4][4];
static cplx SIG[4][4][4][4];    /* sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] */
static int gamma_ready = 0;

static void mat4_mul(cplx a[4][4], cplx b[4][4], cplx out[4][4])
{
    for (int i = 0; i < 4; ++i)
        for (int j = 0; j < 4; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 4; ++k) acc += a[i][k] * b[k][j];
            out[i][j] = acc;
        }
}

static void init_gamma(void)
{
    if (gamma_ready) return;
    /* Pauli matrices */
    cplx pauli[3][2][2] = {
        {{0, 1}, {1, 0}},
        {{0, -I}, {I, 0}},
        {{1, 0}, {0, -1}},
    };
    memset(G, 0, sizeof(G));
    for (int k = 0; k < 3; ++k)
        for (int i = 0; i < 2; ++i)
            for (int j = 0; j < 2; ++j) {
                G[k][i][2 + j] = -I * pauli[k][i][j];
                G[k][2 + i][j] = I * pauli[k][i][j];
            }
    for (int i = 0; i < 2; ++i) {
        G[3][i][2 + i] = -1;
        G[3][2 + i][i] = -1;
    }
    cplx t1[4][4], t2[4][4];
    mat4_mul(G[3], G[0], t1);
    mat4_mul(t1, G[1], t2);
    mat4_mul(t2, G[2], G5);
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = 0; nu < 4; ++nu) {
            cplx ab[4][4], ba[4][4];
            mat4_mul(G[mu], G[nu], ab);
            mat4_mul(G[nu], G[mu], ba);
            for (int i = 0; i < 4; ++i)
                for (int j = 0; j < 4; ++j)
                    SIG[mu][nu][i][j] = 0.5 * I * (ab[i][j] - ba[i][j]);
        }
    gamma_ready = 1;
}

/* gamma_x, gamma_y, gamma_z, gamma_t, gamma_5 as 5 consecutive 4x4 blocks */
void or_gamma(cplx *out)
{
    init_gamma();
    for (int mu = 0; mu < 4; ++mu) memcpy(out + 16 * mu, G[mu], 16 * sizeof(cplx));
    memcpy(out + 64, G5, 16 * sizeof(cplx));
}

/* sigma_{mu nu}, [mu][nu][4][4] */
void or_sigma(cplx *out)
{
    init_gamma();
    memcpy(out, SIG, sizeof(SIG));
}

int or_threads(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 1;
#endif
}

/* thread count of the parallel loops that follow (n >= 1); the arithmetic of
 * every loop is per site, so the results do not depend on it */
void or_set_threads(int n)
{
#ifdef _OPENMP
    if (n >= 1) omp_set_num_threads(n);
#else
    (void)n;
#endif
}

/* ------------------------------------------------------------------ */
/* 3x3 colour algebra                                                   */
/* ------------------------------------------------------------------ */

static const cplx *link_ptr(const cplx *U, long s, int mu) { return U + (s * 4 + mu) * 9; }

static void m3_copy(const cplx *a, cplx *out) { memcpy(out, a, 9 * sizeof(cplx)); }

static void m3_dag(const cplx *a, cplx *out)
{
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) out[i * 3 + j] = conj(a[j * 3 + i]);
}

static void m3_mul(const cplx *a, const cplx *b, cplx *out)
{
    cplx t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cplx acc = 0;
            for (int k = 0; k < 3; ++k) acc += a[i * 3 + k] * b[k * 3 + j];
            t[i * 3 + j] = acc;
        }
    memcpy(out, t, sizeof(t));
}

static void m3_identity(cplx *out)
{
    for (int i = 0; i < 9; ++i) out[i] = (i % 4 == 0) ? 1.0 : 0.0;
}

/* ------------------------------------------------------------------ */
/* clover leaves                                                        */
/* ------------------------------------------------------------------ */

/* One factor of a leaf: the link U_dir(site), daggered or not. */
typedef struct { long site; int dir; int dag; } factor_t;

/*
 * The four leaves of Q_{mu nu}(x), each a closed path from x back to x
 * traversed in the same (mu then nu) orientation:
 *   L0 = U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
 *   L1 = U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
 *   L2 = U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
 *   L3 = U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
 */
static void leaf_factors(long x, int mu, int nu, const int *L, factor_t f[4][4])
{
    int d[4];
#define AT(dm, dn) (memset(d, 0, sizeof(d)), d[mu] += (dm), d[nu] += (dn), shifted(x, L, d))
    long x0 = x;
    long xpm = AT(1, 0), xpn = AT(0, 1), xmm = AT(-1, 0), xmn = AT(0, -1);
    long xmmpn = AT(-1, 1), xmmmn = AT(-1, -1), xmnpm = AT(1, -1);
#undef AT
    factor_t l0[4] = {{x0, mu, 0}, {xpm, nu, 0}, {xpn, mu, 1}, {x0, nu, 1}};
    factor_t l1[4] = {{x0, nu, 0}, {xmmpn, mu, 1}, {xmm, nu, 1}, {xmm, mu, 0}};
    factor_t l2[4] = {{xmm, mu, 1}, {xmmmn, nu, 1}, {xmmmn, mu, 0}, {xmn, nu, 0}};
    factor_t l3[4] = {{xmn, nu, 1}, {xmn, mu, 0}, {xmnpm, nu, 0}, {x0, mu, 1}};
    memcpy(f[0], l0, sizeof(l0));
    memcpy(f[1], l1, sizeof(l1));
    memcpy(f[2], l2, sizeof(l2));
    memcpy(f[3], l3, sizeof(l3));
}

static void factor_matrix(const cplx *U, factor_t f, cplx *out)
{
    if (f.dag) m3_dag(link_ptr(U, f.site, f.dir), out);
    else m3_copy(link_ptr(U, f.site, f.dir), out);
}

/* Q_{mu nu}(x): sum of the four leaves */
static void clover_q(const int *L, const cplx *U, long x, int mu, int nu, cplx *Q)
{
    factor_t f[4][4];
    leaf_factors(x, mu, nu, L, f);
    for (int i = 0; i < 9; ++i) Q[i] = 0;
    for (int l = 0; l < 4; ++l) {
        cplx P[9], A[9];
        m3_identity(P);
        for (int k = 0; k < 4; ++k) {
            factor_matrix(U, f[l][k], A);
            m3_mul(P, A, P);
        }
        for (int i = 0; i < 9; ++i) Q[i] += P[i];
    }
}

/* F_{mu nu}(x) = (Q - Q^dagger) / 8 for the six planes mu < nu, in the order
 * (0,1), (0,2), (0,3), (1,2), (1,3), (2,3) */
void or_field_strength_site(const int *L, const cplx *U, long x, cplx *F6)
{
    int p = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++p) {
            cplx Q[9], Qd[9];
            clover_q(L, U, x, mu, nu, Q);
            m3_dag(Q, Qd);
            for (int i = 0; i < 9; ++i) F6[p * 9 + i] = (Q[i] - Qd[i]) / 8.0;
        }
}

/* C(x) = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} (x) F_{mu nu}(x), 12x12 */
void or_clover_site(const int *L, double kappa, double csw, const cplx *U, long x, cplx *C)
{
    init_gamma();
    cplx F6[54];
    or_field_strength_site(L, U, x, F6);
    for (int i = 0; i < 144; ++i) C[i] = 0;
    for (int i = 0; i < 12; ++i) C[i * 12 + i] = 1;
    int p = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++p)
            for (int s = 0; s < 4; ++s)
                for (int t = 0; t < 4; ++t)
                    for (int a = 0; a < 3; ++a)
                        for (int b = 0; b < 3; ++b)
                            C[(s * 3 + a) * 12 + (t * 3 + b)] +=
                                I * kappa * csw * SIG[mu][nu][s][t] * F6[p * 9 + a * 3 + b];
}

void or_clover_build(const int *L, double kappa, double csw, const cplx *U, cplx *C)
{
    init_gamma();
    long V = vol4(L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) or_clover_site(L, kappa, csw, U, x, C + x * 144);
}

/* inverse of an n x n matrix by Gauss-Jordan elimination with partial
 * pivoting; returns 0 on success, 1 if a pivot is exactly zero */
int or_invert(int n, const cplx *A, cplx *Ainv)
{
    cplx *M = malloc(sizeof(cplx) * n * 2 * n);
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < 2 * n; ++j)
            M[i * 2 * n + j] = (j < n) ? A[i * n + j] : ((j - n == i) ? 1.0 : 0.0);
    for (int c = 0; c < n; ++c) {
        int piv = c;
        for (int r = c + 1; r < n; ++r)
            if (cabs(M[r * 2 * n + c]) > cabs(M[piv * 2 * n + c])) piv = r;
        if (M[piv * 2 * n + c] == 0) { free(M); return 1; }
        if (piv != c)
            for (int j = 0; j < 2 * n; ++j) {
                cplx t = M[c * 2 * n + j];
                M[c * 2 * n + j] = M[piv * 2 * n + j];
                M[piv * 2 * n + j] = t;
            }
        cplx d = M[c * 2 * n + c];
        for (int j = 0; j < 2 * n; ++j) M[c * 2 * n + j] /= d;
        for (int r = 0; r < n; ++r) {
            if (r == c) continue;
            cplx f = M[r * 2 * n + c];
            if (f == 0) continue;
            for (int j = 0; j < 2 * n; ++j) M[r * 2 * n + j] -= f * M[c * 2 * n + j];
        }
    }
    for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) Ainv[i * n + j] = M[i * 2 * n + n + j];
    free(M);
    return 0;
}

int or_clover_invert(const int *L, const cplx *C, cplx *Cinv)
{
    long V = vol4(L);
    int bad = 0;
#pragma omp parallel for schedule(static) reduction(+ : bad)
    for (long x = 0; x < V; ++x) bad += or_invert(12, C + x * 144, Cinv + x * 144);
    return bad;
}

/* ------------------------------------------------------------------ */
/* the Dirac operator                                                   */
/* ------------------------------------------------------------------ */

/*
 * acc -= kappa * sign * (1 + pm * gamma_mu) v, with v = (colour matrix) psi
 * already applied; pm = -1 gives the projector 1 - gamma_mu.
 */
static void add_hop(cplx acc[12], int mu, double pm, double coef, cplx v[4][3])
{
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx gv = 0;
            for (int t = 0; t < 4; ++t) gv += G[mu][s][t] * v[t][a];
            acc[s * 3 + a] -= coef * (v[s][a] + pm * gv);
        }
}

/* v[s] = M psi[s] (M a 3x3 colour matrix, or its adjoint if dag) */
static void colour_apply(const cplx *M, int dag, const cplx *psi, cplx v[4][3])
{
    for (int s = 0; s < 4; ++s)
        for (int a = 0; a < 3; ++a) {
            cplx acc = 0;
            for (int b = 0; b < 3; ++b)
                acc += (dag ? conj(M[b * 3 + a]) : M[a * 3 + b]) * psi[s * 3 + b];
            v[s][a] = acc;
        }
}

/*
 * (D psi)(x) or (D^dagger psi)(x) at one site, given the 12x12 clover C(x).
 * D^dagger is the plain adjoint: C(x)^dagger and the projectors swapped.
 */
static void dirac_site(const int *L, int tbc, double kappa, const cplx *U, const cplx *Cx,
                       const cplx *in, long x, int dagger, cplx out[12])
{
    init_gamma();
    cplx acc[12];
    for (int i = 0; i < 12; ++i) {
        cplx a = 0;
        for (int j = 0; j < 12; ++j)
            a += (dagger ? conj(Cx[j * 12 + i]) : Cx[i * 12 + j]) * in[x * 12 + j];
        acc[i] = a;
    }
    for (int mu = 0; mu < 4; ++mu) {
        int crossed;
        cplx v[4][3];
        long f = neighbour(x, mu, +1, L, &crossed);
        double sg = (mu == 3 && crossed) ? (double)tbc : 1.0;
        colour_apply(link_ptr(U, x, mu), 0, in + f * 12, v);
        add_hop(acc, mu, dagger ? +1.0 : -1.0, kappa * sg, v);
        long b = neighbour(x, mu, -1, L, &crossed);
        sg = (mu == 3 && crossed) ? (double)tbc : 1.0;
        colour_apply(link_ptr(U, b, mu), 1, in + b * 12, v);
        add_hop(acc, mu, dagger ? -1.0 : +1.0, kappa * sg, v);
    }
    for (int i = 0; i < 12; ++i) out[i] = acc[i];
}

void or_dirac(const int *L, int tbc, double kappa, const cplx *U, const cplx *C,
              const cplx *in, cplx *out, int dagger)
{
    init_gamma();
    long V = vol4(L);
#pragma omp parallel for schedule(static)
    for (long x = 0; x < V; ++x) dirac_site(L, tbc, kappa, U, C + x * 144, in, x, dagger, out + x * 12);
}

/* D (or D^dagger) at n listed sites only, with the clover built on the fly;
 * out[i] is the 12-component result at sites[i] */
void or_dirac_at(const int *L, int tbc, double kappa, double csw, const cplx *U, const cplx *in,
                 long n, const long *sites, cplx *out, int dagger)
{
    init_gamma();
#pragma omp parallel for schedule(static)
    for (long i = 0; i < n; ++i) {
        cplx Cx[144];
        or_clover_site(L, kappa, csw, U, sites[i], Cx);
        dirac_site(L, tbc, kappa, U, Cx, in, sites[i], dagger, out + i * 12);
    }
}

/* ------------------------------------------------------------------ */
/* blocks (SAP domains)                                                 */
/* ------------------------------------------------------------------ */

static long block_volume(const int *Bd) { return (long)Bd[0] * Bd[1] * Bd[2] * Bd[3]; }

/* global site of local (lexicographic) index l of block with coords bc */
static long block_site(const int *L, const int *Bd, const int *bc, long l)
{
    int c[4];
    for (int mu = 0; mu < 4; ++mu) {
        c[mu] = bc[mu] * Bd[mu] + (int)(l % Bd[mu]);
        l /= Bd[mu];
    }
    return site_index(c, L);
}

/*
 * Dirichlet block operator D_B on a block vector in_b (V_B x 12, local
 * lexicographic order): every hop whose unwrapped target coordinate leaves the
 * block is dropped.  No boundary sign can arise inside a block.
 */
static void dirac_block_impl(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U,
                             const cplx *C, int compact, const cplx *in_b, cplx *out_b, int dagger)
{
    init_gamma();
    long VB = block_volume(Bd);
    for (long l = 0; l < VB; ++l) {
        long x = block_site(L, Bd, bc, l);
        int lc[4];
        long t = l;
        for (int mu = 0; mu < 4; ++mu) { lc[mu] = (int)(t % Bd[mu]); t /= Bd[mu]; }
        const cplx *Cx = C + (compact ? l : x) * 144;
        cplx acc[12];
        for (int i = 0; i < 12; ++i) {
            cplx a = 0;
            for (int j = 0; j < 12; ++j)
                a += (dagger ? conj(Cx[j * 12 + i]) : Cx[i * 12 + j]) * in_b[l * 12 + j];
            acc[i] = a;
        }
        for (int mu = 0; mu < 4; ++mu) {
            long stride = 1;
            for (int nu = 0; nu < mu; ++nu) stride *= Bd[nu];
            cplx v[4][3];
            if (lc[mu] + 1 < Bd[mu]) {
                colour_apply(link_ptr(U, x, mu), 0, in_b + (l + stride) * 12, v);
                add_hop(acc, mu, dagger ? +1.0 : -1.0, kappa, v);
            }
            if (lc[mu] - 1 >= 0) {
                int crossed;
                long b = neighbour(x, mu, -1, L, &crossed);
                colour_apply(link_ptr(U, b, mu), 1, in_b + (l - stride) * 12, v);
                add_hop(acc, mu, dagger ? -1.0 : +1.0, kappa, v);
            }
        }
        for (int i = 0; i < 12; ++i) out_b[l * 12 + i] = acc[i];
    }
}

static cplx vdot(long n, const cplx *a, const cplx *b)
{
    cplx acc = 0;
    for (long i = 0; i < n; ++i) acc += conj(a[i]) * b[i];
    return acc;
}

static double vnorm2(long n, const cplx *a)
{
    double acc = 0;
    for (long i = 0; i < n; ++i) acc += creal(a[i]) * creal(a[i]) + cimag(a[i]) * cimag(a[i]);
    return acc;
}

/*
 * Minimal residual on D_B: e = 0, r = r_b; k times: p = D_B r,
 * alpha = <p, r>/<p, p> (<a, b> = a^dagger b; alpha = 0 if <p, p> = 0),
 * e += alpha r, r -= alpha p.  r_out (optional) receives the final residual.
 */
void or_dirac_block(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U,
                    const cplx *C, const cplx *in_b, cplx *out_b, int dagger)
{
    dirac_block_impl(L, Bd, bc, kappa, U, C, 0, in_b, out_b, dagger);
}

static void mr_block_impl(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U,
                          const cplx *C, int compact, const cplx *r_b, cplx *e_b, cplx *r_out, int nmr)
{
    long n = block_volume(Bd) * 12;
    cplx *r = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n);
    memcpy(r, r_b, sizeof(cplx) * n);
    for (long i = 0; i < n; ++i) e_b[i] = 0;
    for (int k = 0; k < nmr; ++k) {
        dirac_block_impl(L, Bd, bc, kappa, U, C, compact, r, p, 0);
        cplx pr = vdot(n, p, r);
        double pp = vnorm2(n, p);
        cplx alpha = (pp > 0) ? pr / pp : 0;
        for (long i = 0; i < n; ++i) {
            e_b[i] += alpha * r[i];
            r[i] -= alpha * p[i];
        }
    }
    if (r_out) memcpy(r_out, r, sizeof(cplx) * n);
    free(r);
    free(p);
}

void or_mr_block(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U,
                 const cplx *C, const cplx *r_b, cplx *e_b, cplx *r_out, int nmr)
{
    mr_block_impl(L, Bd, bc, kappa, U, C, 0, r_b, e_b, r_out, nmr);
}

/* the same MR on one block with the block's clover built on the fly from U
 * (for lattices whose full clover field is too large to hold) */
void or_mr_block_at(const int *L, const int *Bd, const int *bc, double kappa, double csw,
                    const cplx *U, const cplx *r_b, cplx *e_b, int nmr)
{
    long VB = block_volume(Bd);
    cplx *Cb = malloc(sizeof(cplx) * VB * 144);
    for (long l = 0; l < VB; ++l) or_clover_site(L, kappa, csw, U, block_site(L, Bd, bc, l), Cb + l * 144);
    mr_block_impl(L, Bd, bc, kappa, U, Cb, 1, r_b, e_b, NULL, nmr);
    free(Cb);
}

/* kappa H_B v on one block (Dirichlet), as v - D_B v with the clover set to 1 */
static void hop_block(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U, const cplx *v,
                      cplx *out)
{
    long VB = block_volume(Bd), n = VB * 12;
    cplx *one = calloc(VB * 144, sizeof(cplx));
    cplx *t = malloc(sizeof(cplx) * n);
    for (long l = 0; l < VB; ++l)
        for (int i = 0; i < 12; ++i) one[l * 144 + i * 12 + i] = 1;
    dirac_block_impl(L, Bd, bc, kappa, U, one, 1, v, t, 0);
    for (long i = 0; i < n; ++i) out[i] = v[i] - t[i];
    free(one);
    free(t);
}

/* parity of the local (lexicographic) block site l; blocks start at even
 * coordinates, so it is the site's global parity */
static int block_parity(const int *Bd, long l)
{
    int s = 0;
    for (int mu = 0; mu < 4; ++mu) {
        s += (int)(l % Bd[mu]);
        l /= Bd[mu];
    }
    return s & 1;
}

/* out = M in site by site over the block (M = C or C^-1 of the block's sites),
 * only on sites of the given parity (others set to 0) */
static void block_site_mul(const int *L, const int *Bd, const int *bc, const cplx *M, int parity, const cplx *in,
                           cplx *out)
{
    long VB = block_volume(Bd);
    for (long l = 0; l < VB; ++l) {
        const cplx *m = M + block_site(L, Bd, bc, l) * 144;
        for (int i = 0; i < 12; ++i) {
            cplx a = 0;
            if (block_parity(Bd, l) == parity)
                for (int j = 0; j < 12; ++j) a += m[i * 12 + j] * in[l * 12 + j];
            out[l * 12 + i] = a;
        }
    }
}

/*
 * Even-odd preconditioned minimal residual on D_B (the block solver of
 * DD-alphaAMG): with the block's sites split by parity,
 * D_B = [[C_ee, -kappa H_eo], [-kappa H_oe, C_oo]]; nmr MR steps from 0 on the
 * even Schur complement  Dh = C_ee - kappa^2 H_eo C_oo^-1 H_oe  with source
 * rh = r_e + kappa H_eo C_oo^-1 r_o, then e_o = C_oo^-1 (r_o + kappa H_oe e_e).
 */
static void mr_eo_block_impl(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U, const cplx *C,
                             const cplx *Ci, const cplx *r_b, cplx *e_b, int nmr)
{
    long VB = block_volume(Bd), n = VB * 12;
    cplx *t = malloc(sizeof(cplx) * n), *h = malloc(sizeof(cplx) * n), *rho = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *y = malloc(sizeof(cplx) * n), *ee = calloc(n, sizeof(cplx));
    /* rh = r_e + kappa H_eo C_oo^-1 r_o (even sites) */
    block_site_mul(L, Bd, bc, Ci, 1, r_b, t);
    hop_block(L, Bd, bc, kappa, U, t, h);
    for (long l = 0; l < VB; ++l)
        for (int i = 0; i < 12; ++i)
            rho[l * 12 + i] = block_parity(Bd, l) == 0 ? r_b[l * 12 + i] + h[l * 12 + i] : 0;
    for (int k = 0; k < nmr; ++k) {
        /* p = Dh rho = C_ee rho - kappa H_eo C_oo^-1 (kappa H_oe rho) */
        hop_block(L, Bd, bc, kappa, U, rho, h);
        block_site_mul(L, Bd, bc, Ci, 1, h, y);
        hop_block(L, Bd, bc, kappa, U, y, h);
        block_site_mul(L, Bd, bc, C, 0, rho, p);
        for (long l = 0; l < VB; ++l)
            if (block_parity(Bd, l) == 0)
                for (int i = 0; i < 12; ++i) p[l * 12 + i] -= h[l * 12 + i];
        cplx pr = vdot(n, p, rho);
        double pp = vnorm2(n, p);
        cplx alpha = (pp > 0) ? pr / pp : 0;
        for (long i = 0; i < n; ++i) {
            ee[i] += alpha * rho[i];
            rho[i] -= alpha * p[i];
        }
    }
    /* e_o = C_oo^-1 (r_o + kappa H_oe e_e) */
    hop_block(L, Bd, bc, kappa, U, ee, h);
    for (long l = 0; l < VB; ++l)
        for (int i = 0; i < 12; ++i) t[l * 12 + i] = block_parity(Bd, l) == 1 ? r_b[l * 12 + i] + h[l * 12 + i] : 0;
    block_site_mul(L, Bd, bc, Ci, 1, t, y);
    for (long l = 0; l < VB; ++l)
        for (int i = 0; i < 12; ++i) e_b[l * 12 + i] = block_parity(Bd, l) == 0 ? ee[l * 12 + i] : y[l * 12 + i];
    free(t); free(h); free(rho); free(p); free(y); free(ee);
}

void or_mr_eo_block(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U, const cplx *C,
                    const cplx *Ci, const cplx *r_b, cplx *e_b, int nmr)
{
    mr_eo_block_impl(L, Bd, bc, kappa, U, C, Ci, r_b, e_b, nmr);
}

/*
 * n_cy multiplicative SAP sweeps on D x = b, x updated in place.  Each sweep
 * visits colour 0 then colour 1; within a colour every block B gets
 * x_B += MR_k(D_B, (b - D x)|_B).  Blocks of one colour do not touch each
 * other, so the residual of a colour is taken once before its blocks are
 * visited.  Requires L[mu] / Bd[mu] even for every mu.
 */
static void sap_impl(const int *L, const int *Bd, int tbc, double kappa, const cplx *U, const cplx *C,
                     const cplx *Ci, const cplx *b, cplx *x, int ncy, int nmr, int eo)
{
    long V = vol4(L);
    long VB = block_volume(Bd);
    int NB[4];
    long nblk = 1;
    for (int mu = 0; mu < 4; ++mu) { NB[mu] = L[mu] / Bd[mu]; nblk *= NB[mu]; }
    cplx *r = malloc(sizeof(cplx) * V * 12);
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            or_dirac(L, tbc, kappa, U, C, x, r, 0);
            for (long i = 0; i < V * 12; ++i) r[i] = b[i] - r[i];
#pragma omp parallel for schedule(dynamic)
            for (long blk = 0; blk < nblk; ++blk) {
                int bc[4];
                long t = blk;
                for (int mu = 0; mu < 4; ++mu) { bc[mu] = (int)(t % NB[mu]); t /= NB[mu]; }
                if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) continue;
                cplx *rb = malloc(sizeof(cplx) * VB * 12);
                cplx *eb = malloc(sizeof(cplx) * VB * 12);
                for (long l = 0; l < VB; ++l) {
                    long s = block_site(L, Bd, bc, l);
                    for (int i = 0; i < 12; ++i) rb[l * 12 + i] = r[s * 12 + i];
                }
                if (eo) mr_eo_block_impl(L, Bd, bc, kappa, U, C, Ci, rb, eb, nmr);
                else or_mr_block(L, Bd, bc, kappa, U, C, rb, eb, NULL, nmr);
                for (long l = 0; l < VB; ++l) {
                    long s = block_site(L, Bd, bc, l);
                    for (int i = 0; i < 12; ++i) x[s * 12 + i] += eb[l * 12 + i];
                }
                free(rb);
                free(eb);
            }
        }
    free(r);
}

/* ------------------------------------------------------------------ */
/* the clover-preconditioned operator A = C^-1 D and its SAP (Sec. 2)   */
/* ------------------------------------------------------------------ */

/* out = C^-1 in site by site (Ci holds C^-1 per site) */
static void clover_inv_apply(long V, const cplx *Ci, const cplx *in, cplx *out)
{
    for (long x = 0; x < V; ++x)
        for (int i = 0; i < 12; ++i) {
            cplx a = 0;
            for (int j = 0; j < 12; ++j) a += Ci[x * 144 + i * 12 + j] * in[x * 12 + j];
            out[x * 12 + i] = a;
        }
}

/*
 * A psi with A = C^-1 D (QWS's operator, Sec. 2): D applied first, then C^-1
 * at every site.  C is the clover field D uses, Ci its inverse.
 */
void or_apply_A(const int *L, int tbc, double kappa, const cplx *U, const cplx *C, const cplx *Ci,
                const cplx *in, cplx *out)
{
    long V = vol4(L);
    cplx *t = malloc(sizeof(cplx) * V * 12);
    or_dirac(L, tbc, kappa, U, C, in, t, 0);
    clover_inv_apply(V, Ci, t, out);
    free(t);
}

/*
 * nj Jacobi iterations on the domain system A_B e = r_b from e = 0, with
 * A_B = C_B^-1 D_B (Dirichlet D_B) split as 1 - (1 - A_B): each iteration is
 * e <- e + (r_b - A_B e).  The first iteration gives e = r_b.
 */
static void jacobi_block_impl(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U,
                              const cplx *C, const cplx *Ci, int compact, const cplx *r_b, cplx *e_b, int nj)
{
    long VB = block_volume(Bd);
    long n = VB * 12;
    cplx *t = malloc(sizeof(cplx) * n);
    for (long i = 0; i < n; ++i) e_b[i] = 0;
    for (int k = 0; k < nj; ++k) {
        dirac_block_impl(L, Bd, bc, kappa, U, C, compact, e_b, t, 0);
        for (long l = 0; l < VB; ++l) {
            const cplx *ci = Ci + (compact ? l : block_site(L, Bd, bc, l)) * 144;
            for (int i = 0; i < 12; ++i) {
                cplx a = 0;
                for (int j = 0; j < 12; ++j) a += ci[i * 12 + j] * t[l * 12 + j];
                e_b[l * 12 + i] += r_b[l * 12 + i] - a;
            }
        }
    }
    free(t);
}

void or_jacobi_block(const int *L, const int *Bd, const int *bc, double kappa, const cplx *U, const cplx *C,
                     const cplx *Ci, const cplx *r_b, cplx *e_b, int nj)
{
    jacobi_block_impl(L, Bd, bc, kappa, U, C, Ci, 0, r_b, e_b, nj);
}

/* the same Jacobi iterations on one block with the block's C and C^-1 built
 * on the fly from U (for lattices whose full clover field is too large) */
void or_jacobi_block_at(const int *L, const int *Bd, const int *bc, double kappa, double csw, const cplx *U,
                        const cplx *r_b, cplx *e_b, int nj)
{
    long VB = block_volume(Bd);
    cplx *Cb = malloc(sizeof(cplx) * VB * 144);
    cplx *Cib = malloc(sizeof(cplx) * VB * 144);
    for (long l = 0; l < VB; ++l) {
        or_clover_site(L, kappa, csw, U, block_site(L, Bd, bc, l), Cb + l * 144);
        or_invert(12, Cb + l * 144, Cib + l * 144);
    }
    jacobi_block_impl(L, Bd, bc, kappa, U, Cb, Cib, 1, r_b, e_b, nj);
    free(Cb);
    free(Cib);
}

/*
 * n_cy multiplicative SAP sweeps on A x = b (QWS's M_SAP for A, Sec. 2):
 * colour 0 then colour 1, every block B of the colour gets
 * x_B += Jacobi_nj(A_B, (b - A x)|_B).
 */
void or_sap_A(const int *L, const int *Bd, int tbc, double kappa, const cplx *U, const cplx *C, const cplx *Ci,
              const cplx *b, cplx *x, int ncy, int nj)
{
    long V = vol4(L);
    long VB = block_volume(Bd);
    int NB[4];
    long nblk = 1;
    for (int mu = 0; mu < 4; ++mu) { NB[mu] = L[mu] / Bd[mu]; nblk *= NB[mu]; }
    cplx *r = malloc(sizeof(cplx) * V * 12);
    for (int cy = 0; cy < ncy; ++cy)
        for (int colour = 0; colour < 2; ++colour) {
            or_apply_A(L, tbc, kappa, U, C, Ci, x, r);
            for (long i = 0; i < V * 12; ++i) r[i] = b[i] - r[i];
#pragma omp parallel for schedule(dynamic)
            for (long blk = 0; blk < nblk; ++blk) {
                int bc[4];
                long t = blk;
                for (int mu = 0; mu < 4; ++mu) { bc[mu] = (int)(t % NB[mu]); t /= NB[mu]; }
                if (((bc[0] + bc[1] + bc[2] + bc[3]) & 1) != colour) continue;
                cplx *rb = malloc(sizeof(cplx) * VB * 12);
                cplx *eb = malloc(sizeof(cplx) * VB * 12);
                for (long l = 0; l < VB; ++l) {
                    long s = block_site(L, Bd, bc, l);
                    for (int i = 0; i < 12; ++i) rb[l * 12 + i] = r[s * 12 + i];
                }
                jacobi_block_impl(L, Bd, bc, kappa, U, C, Ci, 0, rb, eb, nj);
                for (long l = 0; l < VB; ++l) {
                    long s = block_site(L, Bd, bc, l);
                    for (int i = 0; i < 12; ++i) x[s * 12 + i] += eb[l * 12 + i];
                }
                free(rb);
                free(eb);
            }
        }
    free(r);
}

/*
 * The QWS solver for D x = b (Sec. 2).  With A = C^-1 D the system is
 * A x = C^-1 b.  Richardson iteration: r = C^-1 b - A x; solve
 * (A M_SAP) y = r / ||r|| with BiCGStab to the relative residual inner_tol
 * (M_SAP = n_cy sweeps of or_sap_A from zero with nj Jacobi iterations per
 * block); x += ||r|| M_SAP y; stop when ||b - D x|| <= tol ||b|| (the true
 * residual of D).  BiCGStab on K = A M_SAP from y = 0:
 *   r = rhs, r0 = r, p = r, rho = <r0, r>; then v = K p,
 *   alpha = rho / <r0, v>, s = r - alpha v, t = K s, omega = <t, s>/<t, t>,
 *   y += alpha p + omega s, r = s - omega t, rho' = <r0, r>,
 *   beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v).
 * Returns 0 when converged; *iters counts BiCGStab iterations.
 */
typedef struct {
    const int *L, *Bd;
    int tbc;
    double kappa;
    const cplx *U, *C, *Ci;
    int ncy, nj;
} qws_t;

static void qws_M(const qws_t *q, const cplx *v, cplx *z, long n)
{
    for (long i = 0; i < n; ++i) z[i] = 0;
    or_sap_A(q->L, q->Bd, q->tbc, q->kappa, q->U, q->C, q->Ci, v, z, q->ncy, q->nj);
}

static void qws_K(const qws_t *q, const cplx *v, cplx *out, cplx *tmp, long n)
{
    qws_M(q, v, tmp, n);
    or_apply_A(q->L, q->tbc, q->kappa, q->U, q->C, q->Ci, tmp, out);
}

int or_solve_qws(const int *L, const int *Bd, int tbc, double kappa, const cplx *U, const cplx *C, const cplx *Ci,
                 const cplx *b, cplx *x, int ncy, int nj, double tol, double inner_tol, int max_iter, int *iters_out,
                 double *res_out)
{
    qws_t q = {L, Bd, tbc, kappa, U, C, Ci, ncy, nj};
    long V = vol4(L), n = V * 12;
    cplx *r = malloc(sizeof(cplx) * n), *ra = malloc(sizeof(cplx) * n), *rhs = malloc(sizeof(cplx) * n);
    cplx *y = malloc(sizeof(cplx) * n), *rr = malloc(sizeof(cplx) * n), *r0 = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *v = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n);
    cplx *t = malloc(sizeof(cplx) * n), *tmp = malloc(sizeof(cplx) * n), *e = malloc(sizeof(cplx) * n);
    double bnorm = sqrt(vnorm2(n, b));
    int iters = 0, status = 1;
    double rel = 0;
    if (bnorm == 0) {
        for (long i = 0; i < n; ++i) x[i] = 0;
        status = 0;
        goto done;
    }
    for (;;) {
        /* true residual of D, then the residual of A */
        or_dirac(L, tbc, kappa, U, C, x, tmp, 0);
        for (long i = 0; i < n; ++i) r[i] = b[i] - tmp[i];
        rel = sqrt(vnorm2(n, r)) / bnorm;
        if (rel <= tol) { status = 0; break; }
        if (iters >= max_iter) break;
        clover_inv_apply(V, Ci, r, ra);
        double rn = sqrt(vnorm2(n, ra));
        for (long i = 0; i < n; ++i) rhs[i] = ra[i] / rn;
        /* BiCGStab on (A M) y = rhs */
        for (long i = 0; i < n; ++i) { y[i] = 0; rr[i] = rhs[i]; r0[i] = rhs[i]; p[i] = rhs[i]; }
        cplx rho = vdot(n, r0, rr);
        while (iters < max_iter) {
            qws_K(&q, p, v, tmp, n);
            cplx r0v = vdot(n, r0, v);
            if (r0v == 0) break;
            cplx alpha = rho / r0v;
            for (long i = 0; i < n; ++i) s[i] = rr[i] - alpha * v[i];
            qws_K(&q, s, t, tmp, n);
            double tt = vnorm2(n, t);
            cplx omega = (tt > 0) ? vdot(n, t, s) / tt : 0;
            for (long i = 0; i < n; ++i) {
                y[i] += alpha * p[i] + omega * s[i];
                rr[i] = s[i] - omega * t[i];
            }
            ++iters;
            if (sqrt(vnorm2(n, rr)) <= inner_tol) break;
            cplx rho1 = vdot(n, r0, rr);
            if (rho == 0 || omega == 0) break;
            cplx beta = (rho1 / rho) * (alpha / omega);
            for (long i = 0; i < n; ++i) p[i] = rr[i] + beta * (p[i] - omega * v[i]);
            rho = rho1;
        }
        /* x += ||r|| M y */
        qws_M(&q, y, e, n);
        for (long i = 0; i < n; ++i) x[i] += rn * e[i];
    }
done:
    *iters_out = iters;
    *res_out = rel;
    free(r); free(ra); free(rhs); free(y); free(rr); free(r0); free(p); free(v); free(s); free(t); free(tmp);
    free(e);
    return status;
}

void or_sap(const int *L, const int *Bd, int tbc, double kappa, const cplx *U, const cplx *C,
            const cplx *b, cplx *x, int ncy, int nmr)
{
    sap_impl(L, Bd, tbc, kappa, U, C, NULL, b, x, ncy, nmr, 0);
}

/* the same sweeps with the even-odd preconditioned MR block solver */
void or_sap_eo(const int *L, const int *Bd, int tbc, double kappa, const cplx *U, const cplx *C, const cplx *Ci,
               const cplx *b, cplx *x, int ncy, int nmr)
{
    sap_impl(L, Bd, tbc, kappa, U, C, Ci, b, x, ncy, nmr, 1);
}

/* ------------------------------------------------------------------ */
/* outer solvers                                                        */
/* ------------------------------------------------------------------ */

typedef struct {
    const int *L, *Bd;
    int tbc;
    double kappa;
    const cplx *U, *C;
    int precond; /* 0: identity, 1: SAP */
    int ncy, nmr;
} op_t;

static void op_apply(const op_t *op, const cplx *in, cplx *out)
{
    or_dirac(op->L, op->tbc, op->kappa, op->U, op->C, in, out, 0);
}

/* z = M v: n_cy SAP sweeps from z = 0 with source v (or z = v) */
static void op_precond(const op_t *op, const cplx *v, cplx *z, long n)
{
    if (op->precond == 0) { memcpy(z, v, sizeof(cplx) * n); return; }
    for (long i = 0; i < n; ++i) z[i] = 0;
    or_sap(op->L, op->Bd, op->tbc, op->kappa, op->U, op->C, v, z, op->ncy, op->nmr);
}

static double true_residual(const op_t *op, const cplx *b, const cplx *x, long n, cplx *tmp)
{
    op_apply(op, x, tmp);
    double acc = 0;
    for (long i = 0; i < n; ++i) {
        cplx d = b[i] - tmp[i];
        acc += creal(d) * creal(d) + cimag(d) * cimag(d);
    }
    return sqrt(acc);
}

/*
 * FGCR(m) with right preconditioner M and restarts.  x starts at the value
 * passed in.  Each iteration: z_j = M r, w_j = D z_j, modified Gram-Schmidt of
 * w_j against the normalised w_i (the same combination applied to z_j),
 * normalisation, alpha = <w_j, r>, x += alpha z_j, r -= alpha w_j.  At the end
 * of a cycle, or when ||r|| <= tol ||b||, the residual is recomputed as b - D x;
 * the solve ends when that true residual meets tol.
 * Returns 0 if converged, 1 if max_iter was reached.
 */
static int fgcr(const op_t *op, const cplx *b, cplx *x, int m, double tol, int max_iter,
                int *iters_out, double *res_out)
{
    long n = vol4(op->L) * 12;
    cplx *r = malloc(sizeof(cplx) * n);
    cplx *tmp = malloc(sizeof(cplx) * n);
    cplx **z = malloc(sizeof(cplx *) * m);
    cplx **w = malloc(sizeof(cplx *) * m);
    for (int j = 0; j < m; ++j) {
        z[j] = malloc(sizeof(cplx) * n);
        w[j] = malloc(sizeof(cplx) * n);
    }
    double bnorm = sqrt(vnorm2(n, b));
    int iters = 0, status = 1;
    double rel = 0;
    if (bnorm == 0) {
        for (long i = 0; i < n; ++i) x[i] = 0;
        status = 0;
        goto done;
    }
    op_apply(op, x, tmp);
    for (long i = 0; i < n; ++i) r[i] = b[i] - tmp[i];
    while (iters < max_iter) {
        int j;
        for (j = 0; j < m && iters < max_iter; ++j) {
            op_precond(op, r, z[j], n);
            op_apply(op, z[j], w[j]);
            for (int i = 0; i < j; ++i) {
                cplx beta = vdot(n, w[i], w[j]);
                for (long k = 0; k < n; ++k) {
                    w[j][k] -= beta * w[i][k];
                    z[j][k] -= beta * z[i][k];
                }
            }
            double nw = sqrt(vnorm2(n, w[j]));
            for (long k = 0; k < n; ++k) {
                w[j][k] /= nw;
                z[j][k] /= nw;
            }
            cplx alpha = vdot(n, w[j], r);
            for (long k = 0; k < n; ++k) {
                x[k] += alpha * z[j][k];
                r[k] -= alpha * w[j][k];
            }
            ++iters;
            if (sqrt(vnorm2(n, r)) <= tol * bnorm) { ++j; break; }
        }
        rel = true_residual(op, b, x, n, tmp) / bnorm;
        if (rel <= tol) { status = 0; break; }
        for (long i = 0; i < n; ++i) r[i] = b[i] - tmp[i];
    }
    if (status != 0) rel = true_residual(op, b, x, n, tmp) / bnorm;
done:
    *iters_out = iters;
    *res_out = rel;
    for (int j = 0; j < m; ++j) { free(z[j]); free(w[j]); }
    free(z); free(w); free(r); free(tmp);
    return status;
}

/*
 * Flexible BiCGStab with right preconditioner M (the paper's outer solver,
 * Sec. 3): r = b - D x, r0 = r, p = r, rho = <r0, r>; then
 *   p^ = M p, v = D p^, alpha = rho / <r0, v>, s = r - alpha v,
 *   s^ = M s, t = D s^, omega = <t, s>/<t, t>,
 *   x += alpha p^ + omega s^, r = s - omega t,
 *   rho' = <r0, r>, beta = (rho'/rho)(alpha/omega), p = r + beta (p - omega v).
 * The true residual is checked when the recursive one meets tol.
 */
static int fbicgstab(const op_t *op, const cplx *b, cplx *x, double tol, int max_iter,
                     int *iters_out, double *res_out)
{
    long n = vol4(op->L) * 12;
    cplx *r = malloc(sizeof(cplx) * n), *r0 = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *ph = malloc(sizeof(cplx) * n);
    cplx *v = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n);
    cplx *sh = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *tmp = malloc(sizeof(cplx) * n);
    double bnorm = sqrt(vnorm2(n, b));
    int iters = 0, status = 1;
    double rel = 0;
    if (bnorm == 0) {
        for (long i = 0; i < n; ++i) x[i] = 0;
        status = 0;
        goto done;
    }
    for (;;) {
        op_apply(op, x, tmp);
        for (long i = 0; i < n; ++i) { r[i] = b[i] - tmp[i]; r0[i] = r[i]; p[i] = r[i]; }
        cplx rho = vdot(n, r0, r);
        int restart = 0;
        while (iters < max_iter) {
            op_precond(op, p, ph, n);
            op_apply(op, ph, v);
            cplx r0v = vdot(n, r0, v);
            if (r0v == 0) { restart = 1; break; }
            cplx alpha = rho / r0v;
            for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
            op_precond(op, s, sh, n);
            op_apply(op, sh, t);
            double tt = vnorm2(n, t);
            cplx omega = (tt > 0) ? vdot(n, t, s) / tt : 0;
            for (long i = 0; i < n; ++i) {
                x[i] += alpha * ph[i] + omega * sh[i];
                r[i] = s[i] - omega * t[i];
            }
            ++iters;
            if (sqrt(vnorm2(n, r)) <= tol * bnorm) break;
            cplx rho1 = vdot(n, r0, r);
            if (rho == 0 || omega == 0) { restart = 1; break; }
            cplx beta = (rho1 / rho) * (alpha / omega);
            for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            rho = rho1;
        }
        rel = true_residual(op, b, x, n, tmp) / bnorm;
        if (rel <= tol) { status = 0; break; }
        if (iters >= max_iter) break;
        (void)restart;
    }
done:
    *iters_out = iters;
    *res_out = rel;
    free(r); free(r0); free(p); free(ph); free(v); free(s); free(sh); free(t); free(tmp);
    return status;
}

/*
 * Solve D x = b (x holds the initial guess on entry).  method 0: FGCR(m);
 * method 1: flexible BiCGStab.  precond 0: none; 1: n_cy SAP sweeps with
 * n_mr MR steps per block.  Returns 0 when ||b - D x|| <= tol ||b||.
 */
int or_solve(const int *L, const int *Bd, int tbc, double kappa, const cplx *U, const cplx *C,
             const cplx *b, cplx *x, int method, int precond, int ncy, int nmr, int m,
             double tol, int max_iter, int *iters, double *true_res)
{
    op_t op = {L, Bd, tbc, kappa, U, C, precond, ncy, nmr};
    if (method == 0) return fgcr(&op, b, x, m, tol, max_iter, iters, true_res);
    return fbicgstab(&op, b, x, tol, max_iter, iters, true_res);
}

/* ------------------------------------------------------------------ */
/* two-level multigrid (Sec. 3)                                          */
/* ------------------------------------------------------------------ */

/*
 * Aggregates are blocks of Ad[0] x Ad[1] x Ad[2] x Ad[3] fine sites; the
 * coarse lattice has Lc = L / Ad sites, indexed lexicographically (x fastest).
 * Each aggregate is split by chirality (chi = 0: spins 0, 1, components 0..5;
 * chi = 1: spins 2, 3, components 6..11), so a coarse site carries 2 nvec
 * degrees of freedom, ordered (chi, i).  A coarse vector is u[a][chi][i].
 * W holds nvec fine fields [i][site][12], orthonormal within every
 * (aggregate, chirality): P u = sum_i W_i u(a(x), chi, i), R = P^dagger.
 * The coarse operator D_c = R D P is stored as a 9-point stencil
 * Dc[a][k][(chi', j)][(chi, i)], k = 0 for the coupling inside the aggregate
 * (clover term and hops that stay inside), k = 1 + 2 mu for the fine hops from
 * x + mu that cross the aggregate's +mu face, k = 2 + 2 mu for those from x - mu
 * across its -mu face; (D_c u)(a) = sum_k Dc[a][k] u(a + offset_k).
 */
static void coarse_dims(const int *L, const int *Ad, int Lc[4])
{
    for (int mu = 0; mu < 4; ++mu) Lc[mu] = L[mu] / Ad[mu];
}

static long agg_of(long x, const int *L, const int *Ad)
{
    int c[4], Lc[4];
    site_coords(x, L, c);
    coarse_dims(L, Ad, Lc);
    for (int mu = 0; mu < 4; ++mu) c[mu] /= Ad[mu];
    return site_index(c, Lc);
}

/* coarse neighbour of a for stencil index k (k = 0: a itself) */
static long coarse_nbr(long a, int k, const int *Lc)
{
    if (k == 0) return a;
    int mu = (k - 1) / 2, dir = ((k - 1) % 2 == 0) ? +1 : -1, crossed;
    return neighbour(a, mu, dir, Lc, &crossed);
}

/*
 * Block modified Gram-Schmidt: for every aggregate and chirality, the
 * restrictions of V_0 .. V_{nvec-1} are orthonormalised in order.  Returns the
 * number of restrictions that were linearly dependent (zero after projection).
 */
int or_mg_basis(const int *L, const int *Ad, int nvec, const cplx *Vin, cplx *W)
{
    long V = vol4(L);
    memcpy(W, Vin, sizeof(cplx) * nvec * V * 12);
    int Lc[4];
    coarse_dims(L, Ad, Lc);
    long Vc = vol4(Lc), VA = V / Vc;
    /* the sites of every aggregate, in increasing site order */
    long *sites = malloc(sizeof(long) * V), *fill = calloc(Vc, sizeof(long));
    for (long x = 0; x < V; ++x) {
        long a = agg_of(x, L, Ad);
        sites[a * VA + fill[a]++] = x;
    }
    int bad = 0;
    for (long a = 0; a < Vc; ++a)
        for (int chi = 0; chi < 2; ++chi)
            for (int i = 0; i < nvec; ++i) {
                cplx *wi = W + (long)i * V * 12;
                const long *sa = sites + a * VA;
                for (int j = 0; j < i; ++j) {
                    const cplx *wj = W + (long)j * V * 12;
                    cplx d = 0;
                    for (long q = 0; q < VA; ++q)
                        for (int c = 6 * chi; c < 6 * chi + 6; ++c) d += conj(wj[sa[q] * 12 + c]) * wi[sa[q] * 12 + c];
                    for (long q = 0; q < VA; ++q)
                        for (int c = 6 * chi; c < 6 * chi + 6; ++c) wi[sa[q] * 12 + c] -= d * wj[sa[q] * 12 + c];
                }
                double n2 = 0;
                for (long q = 0; q < VA; ++q)
                    for (int c = 6 * chi; c < 6 * chi + 6; ++c) {
                        cplx z = wi[sa[q] * 12 + c];
                        n2 += creal(z) * creal(z) + cimag(z) * cimag(z);
                    }
                if (n2 == 0) { ++bad; continue; }
                double inv = 1.0 / sqrt(n2);
                for (long q = 0; q < VA; ++q)
                    for (int c = 6 * chi; c < 6 * chi + 6; ++c) wi[sa[q] * 12 + c] *= inv;
            }
    free(sites);
    free(fill);
    return bad;
}

/* u = R v = P^dagger v */
void or_mg_restrict(const int *L, const int *Ad, int nvec, const cplx *W, const cplx *v, cplx *u)
{
    long V = vol4(L);
    int Lc[4];
    coarse_dims(L, Ad, Lc);
    long nc = vol4(Lc) * 2 * nvec;
    for (long k = 0; k < nc; ++k) u[k] = 0;
    for (long x = 0; x < V; ++x) {
        long a = agg_of(x, L, Ad);
        for (int chi = 0; chi < 2; ++chi)
            for (int i = 0; i < nvec; ++i) {
                const cplx *wi = W + (long)i * V * 12;
                cplx d = 0;
                for (int c = 6 * chi; c < 6 * chi + 6; ++c) d += conj(wi[x * 12 + c]) * v[x * 12 + c];
                u[(a * 2 + chi) * nvec + i] += d;
            }
    }
}

/* v = P u */
void or_mg_prolong(const int *L, const int *Ad, int nvec, const cplx *W, const cplx *u, cplx *v)
{
    long V = vol4(L);
    for (long x = 0; x < V; ++x) {
        long a = agg_of(x, L, Ad);
        for (int c = 0; c < 12; ++c) {
            int chi = c / 6;
            cplx acc = 0;
            for (int i = 0; i < nvec; ++i) acc += W[(long)i * V * 12 + x * 12 + c] * u[(a * 2 + chi) * nvec + i];
            v[x * 12 + c] = acc;
        }
    }
}

/* the hop term of D at x from its neighbour in direction dir (+1/-1) along mu:
 * -kappa s (1 -/+ gamma_mu) U psi(y), s the boundary sign (out is overwritten) */
static void hop_term(const int *L, int tbc, double kappa, const cplx *U, long x, int mu, int dir, const cplx *psi_y,
                     cplx out[12])
{
    init_gamma();
    int crossed;
    long y = neighbour(x, mu, dir, L, &crossed);
    double sg = (mu == 3 && crossed) ? (double)tbc : 1.0;
    cplx v[4][3];
    if (dir > 0) colour_apply(link_ptr(U, x, mu), 0, psi_y, v);
    else colour_apply(link_ptr(U, y, mu), 1, psi_y, v);
    for (int i = 0; i < 12; ++i) out[i] = 0;
    add_hop(out, mu, dir > 0 ? -1.0 : +1.0, kappa * sg, v);
}

/* Dc = R D P, assembled per fine site and hop direction (layout above) */
void or_mg_coarse_op(const int *L, const int *Ad, int tbc, double kappa, const cplx *U, const cplx *C, int nvec,
                     const cplx *W, cplx *Dc)
{
    long V = vol4(L);
    int Lc[4];
    coarse_dims(L, Ad, Lc);
    long Vc = vol4(Lc);
    const int N2 = 2 * nvec;
    memset(Dc, 0, sizeof(cplx) * Vc * 9 * N2 * N2);
    for (long x = 0; x < V; ++x) {
        long a = agg_of(x, L, Ad);
        int c[4];
        site_coords(x, L, c);
        for (int k = 0; k < 9; ++k) {
            /* the pieces of D at x that belong to stencil entry k */
            for (int chi = 0; chi < 2; ++chi)
                for (int i = 0; i < nvec; ++i) {
                    const cplx *wi = W + (long)i * V * 12;
                    cplx h[12] = {0};
                    if (k == 0) {
                        /* clover term, then the hops that stay inside the aggregate */
                        cplx p[12];
                        for (int q = 0; q < 12; ++q) p[q] = (q / 6 == chi) ? wi[x * 12 + q] : 0;
                        for (int r = 0; r < 12; ++r)
                            for (int q = 0; q < 12; ++q) h[r] += C[x * 144 + r * 12 + q] * p[q];
                        for (int mu = 0; mu < 4; ++mu)
                            for (int dir = -1; dir <= 1; dir += 2) {
                                int inside = (dir > 0) ? ((c[mu] + 1) % Ad[mu] != 0) : (c[mu] % Ad[mu] != 0);
                                if (!inside) continue;
                                int crossed;
                                long y = neighbour(x, mu, dir, L, &crossed);
                                for (int q = 0; q < 12; ++q) p[q] = (q / 6 == chi) ? wi[y * 12 + q] : 0;
                                cplx t[12];
                                hop_term(L, tbc, kappa, U, x, mu, dir, p, t);
                                for (int r = 0; r < 12; ++r) h[r] += t[r];
                            }
                    } else {
                        int mu = (k - 1) / 2, dir = ((k - 1) % 2 == 0) ? +1 : -1;
                        int across = (dir > 0) ? ((c[mu] + 1) % Ad[mu] == 0) : (c[mu] % Ad[mu] == 0);
                        if (!across) continue;
                        int crossed;
                        long y = neighbour(x, mu, dir, L, &crossed);
                        cplx p[12];
                        for (int q = 0; q < 12; ++q) p[q] = (q / 6 == chi) ? wi[y * 12 + q] : 0;
                        hop_term(L, tbc, kappa, U, x, mu, dir, p, h);
                    }
                    for (int chp = 0; chp < 2; ++chp)
                        for (int j = 0; j < nvec; ++j) {
                            const cplx *wj = W + (long)j * V * 12;
                            cplx d = 0;
                            for (int q = 6 * chp; q < 6 * chp + 6; ++q) d += conj(wj[x * 12 + q]) * h[q];
                            Dc[((a * 9 + k) * N2 + chp * nvec + j) * N2 + chi * nvec + i] += d;
                        }
                }
        }
    }
}

void or_mg_coarse_apply(const int *L, const int *Ad, int nvec, const cplx *Dc, const cplx *u, cplx *out)
{
    int Lc[4];
    coarse_dims(L, Ad, Lc);
    long Vc = vol4(Lc);
    const int N2 = 2 * nvec;
    for (long a = 0; a < Vc; ++a)
        for (int r = 0; r < N2; ++r) {
            cplx acc = 0;
            for (int k = 0; k < 9; ++k) {
                long b = coarse_nbr(a, k, Lc);
                for (int q = 0; q < N2; ++q) acc += Dc[((a * 9 + k) * N2 + r) * N2 + q] * u[b * N2 + q];
            }
            out[a * N2 + r] = acc;
        }
}

/* BiCGStab on D_c x = b from x = 0 to ||r|| <= tol ||b|| or maxit iterations */
int or_mg_coarse_solve(const int *L, const int *Ad, int nvec, const cplx *Dc, const cplx *b, cplx *x, double tol,
                       int maxit, int *iters_out)
{
    int Lc[4];
    coarse_dims(L, Ad, Lc);
    long n = vol4(Lc) * 2 * nvec;
    cplx *r = malloc(sizeof(cplx) * n), *r0 = malloc(sizeof(cplx) * n), *p = malloc(sizeof(cplx) * n);
    cplx *v = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    double bn = sqrt(vnorm2(n, b));
    int it = 0, status = 1;
    for (long i = 0; i < n; ++i) { x[i] = 0; r[i] = b[i]; r0[i] = b[i]; p[i] = b[i]; }
    if (bn == 0) { status = 0; goto done; }
    cplx rho = vdot(n, r0, r);
    while (it < maxit) {
        or_mg_coarse_apply(L, Ad, nvec, Dc, p, v);
        cplx r0v = vdot(n, r0, v);
        if (r0v == 0) break;
        cplx alpha = rho / r0v;
        for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
        or_mg_coarse_apply(L, Ad, nvec, Dc, s, t);
        double tt = vnorm2(n, t);
        cplx omega = (tt > 0) ? vdot(n, t, s) / tt : 0;
        for (long i = 0; i < n; ++i) {
            x[i] += alpha * p[i] + omega * s[i];
            r[i] = s[i] - omega * t[i];
        }
        ++it;
        if (sqrt(vnorm2(n, r)) <= tol * bn) { status = 0; break; }
        cplx rho1 = vdot(n, r0, r);
        if (rho == 0 || omega == 0) break;
        cplx beta = (rho1 / rho) * (alpha / omega);
        for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
        rho = rho1;
    }
done:
    *iters_out = it;
    free(r); free(r0); free(p); free(v); free(s); free(t);
    return status;
}

typedef struct {
    const int *L, *Bd, *Ad;
    int tbc;
    double kappa;
    const cplx *U, *C, *Ci;
    int nvec;
    const cplx *W, *Dc;
    int ncy, nj;     /* post-smoother: n_cy sweeps of the SAP for A, nj Jacobi iterations */
    double ctol;     /* coarse BiCGStab tolerance and iteration limit */
    int cmaxit;
} mg_t;

/*
 * One application of the two-level preconditioner to v: the coarse-grid
 * correction x = P D_c^-1 R v (D_c^-1 by BiCGStab to ctol), then the
 * post-smoother x += M_SAP(C^-1 (v - D x)) with QWS's M_SAP for A (Sec. 3).
 */
static void mg_apply(const mg_t *m, const cplx *v, cplx *x)
{
    long V = vol4(m->L), n = V * 12;
    int Lc[4];
    coarse_dims(m->L, m->Ad, Lc);
    long nc = vol4(Lc) * 2 * m->nvec;
    cplx *u = malloc(sizeof(cplx) * nc), *cx = malloc(sizeof(cplx) * nc);
    cplx *r = malloc(sizeof(cplx) * n), *ra = malloc(sizeof(cplx) * n), *e = malloc(sizeof(cplx) * n);
    int it;
    or_mg_restrict(m->L, m->Ad, m->nvec, m->W, v, u);
    or_mg_coarse_solve(m->L, m->Ad, m->nvec, m->Dc, u, cx, m->ctol, m->cmaxit, &it);
    or_mg_prolong(m->L, m->Ad, m->nvec, m->W, cx, x);
    or_dirac(m->L, m->tbc, m->kappa, m->U, m->C, x, r, 0);
    for (long i = 0; i < n; ++i) r[i] = v[i] - r[i];
    clover_inv_apply(V, m->Ci, r, ra);
    for (long i = 0; i < n; ++i) e[i] = 0;
    or_sap_A(m->L, m->Bd, m->tbc, m->kappa, m->U, m->C, m->Ci, ra, e, m->ncy, m->nj);
    for (long i = 0; i < n; ++i) x[i] += e[i];
    free(u); free(cx); free(r); free(ra); free(e);
}

void or_mg_precond(const int *L, const int *Bd, const int *Ad, int tbc, double kappa, const cplx *U, const cplx *C,
                   const cplx *Ci, int nvec, const cplx *W, const cplx *Dc, int ncy, int nj, double ctol, int cmaxit,
                   const cplx *v, cplx *x)
{
    mg_t m = {L, Bd, Ad, tbc, kappa, U, C, Ci, nvec, W, Dc, ncy, nj, ctol, cmaxit};
    mg_apply(&m, v, x);
}

/*
 * Setup (Sec. 3): the initial null vectors are M_SAP applied to nvec random
 * vectors eta (given), V_i = M_SAP(C^-1 eta_i); W and D_c are built from them;
 * then n_adapt times every V_i is replaced by the two-level preconditioner
 * (with the current W, D_c) applied to it, and W, D_c are rebuilt.  Returns
 * the number of linearly dependent aggregate restrictions met.
 */
int or_mg_setup(const int *L, const int *Bd, const int *Ad, int tbc, double kappa, const cplx *U, const cplx *C,
                const cplx *Ci, int nvec, const cplx *eta, int ncy, int nj, int n_adapt, double ctol, int cmaxit,
                cplx *W, cplx *Dc)
{
    long V = vol4(L), n = V * 12;
    cplx *Vv = malloc(sizeof(cplx) * nvec * n), *ra = malloc(sizeof(cplx) * n);
    for (int i = 0; i < nvec; ++i) {
        clover_inv_apply(V, Ci, eta + (long)i * n, ra);
        cplx *vi = Vv + (long)i * n;
        for (long k = 0; k < n; ++k) vi[k] = 0;
        or_sap_A(L, Bd, tbc, kappa, U, C, Ci, ra, vi, ncy, nj);
    }
    int bad = or_mg_basis(L, Ad, nvec, Vv, W);
    or_mg_coarse_op(L, Ad, tbc, kappa, U, C, nvec, W, Dc);
    mg_t m = {L, Bd, Ad, tbc, kappa, U, C, Ci, nvec, W, Dc, ncy, nj, ctol, cmaxit};
    cplx *t = malloc(sizeof(cplx) * n);
    for (int pass = 0; pass < n_adapt; ++pass) {
        for (int i = 0; i < nvec; ++i) {
            mg_apply(&m, Vv + (long)i * n, t);
            memcpy(Vv + (long)i * n, t, sizeof(cplx) * n);
        }
        bad += or_mg_basis(L, Ad, nvec, Vv, W);
        or_mg_coarse_op(L, Ad, tbc, kappa, U, C, nvec, W, Dc);
    }
    free(t); free(Vv); free(ra);
    return bad;
}

/*
 * The multigrid solve of D x = b (Sec. 3): flexible BiCGStab (the outer solver
 * of the paper) with the two-level preconditioner, from x = 0, stopping when
 * the true residual ||b - D x|| <= tol ||b||.  Returns 0 when converged.
 */
int or_solve_mg(const int *L, const int *Bd, const int *Ad, int tbc, double kappa, const cplx *U, const cplx *C,
                const cplx *Ci, int nvec, const cplx *W, const cplx *Dc, int ncy, int nj, double ctol, int cmaxit,
                const cplx *b, cplx *x, double tol, int max_iter, int *iters_out, double *res_out)
{
    mg_t m = {L, Bd, Ad, tbc, kappa, U, C, Ci, nvec, W, Dc, ncy, nj, ctol, cmaxit};
    long n = vol4(L) * 12;
    cplx *r = malloc(sizeof(cplx) * n), *r0 = malloc(sizeof(cplx) * n);
    cplx *p = malloc(sizeof(cplx) * n), *ph = malloc(sizeof(cplx) * n);
    cplx *v = malloc(sizeof(cplx) * n), *s = malloc(sizeof(cplx) * n);
    cplx *sh = malloc(sizeof(cplx) * n), *t = malloc(sizeof(cplx) * n);
    cplx *tmp = malloc(sizeof(cplx) * n);
    double bnorm = sqrt(vnorm2(n, b));
    int iters = 0, status = 1;
    double rel = 0;
    for (long i = 0; i < n; ++i) x[i] = 0;
    if (bnorm == 0) { status = 0; goto done; }
    for (;;) {
        or_dirac(L, tbc, kappa, U, C, x, tmp, 0);
        for (long i = 0; i < n; ++i) { r[i] = b[i] - tmp[i]; r0[i] = r[i]; p[i] = r[i]; }
        rel = sqrt(vnorm2(n, r)) / bnorm;
        if (rel <= tol) { status = 0; break; }
        if (iters >= max_iter) break;
        cplx rho = vdot(n, r0, r);
        while (iters < max_iter) {
            mg_apply(&m, p, ph);
            or_dirac(L, tbc, kappa, U, C, ph, v, 0);
            cplx r0v = vdot(n, r0, v);
            if (r0v == 0) break;
            cplx alpha = rho / r0v;
            for (long i = 0; i < n; ++i) s[i] = r[i] - alpha * v[i];
            mg_apply(&m, s, sh);
            or_dirac(L, tbc, kappa, U, C, sh, t, 0);
            double tt = vnorm2(n, t);
            cplx omega = (tt > 0) ? vdot(n, t, s) / tt : 0;
            for (long i = 0; i < n; ++i) {
                x[i] += alpha * ph[i] + omega * sh[i];
                r[i] = s[i] - omega * t[i];
            }
            ++iters;
            if (sqrt(vnorm2(n, r)) <= tol * bnorm) break;
            cplx rho1 = vdot(n, r0, r);
            if (rho == 0 || omega == 0) break;
            cplx beta = (rho1 / rho) * (alpha / omega);
            for (long i = 0; i < n; ++i) p[i] = r[i] + beta * (p[i] - omega * v[i]);
            rho = rho1;
        }
    }
done:
    *iters_out = iters;
    *res_out = rel;
    free(r); free(r0); free(p); free(ph); free(v); free(s); free(sh); free(t); free(tmp);
    return status;
}

/* ------------------------------------------------------------------ */
/* force                                                                */
/* ------------------------------------------------------------------ */

/*
 * dS/dU for S = ||Y||^2, Y = D^-dagger phi, X = D^-1 Y (X and Y given).
 * delta S = -2 Re Y^dagger (delta D) X, delta D = -kappa delta H + delta C.
 * The tensor returned per link, g = dS/dRe U + i dS/dIm U, satisfies
 * delta S = Re sum_ab conj(g_ab) delta U_ab.
 *
 * Hopping part, from the two hops that carry U_mu(x):
 *   g += 2 kappa s [ sum_s ((1-gamma_mu) Y(x))_s X(x+mu)_s^dagger
 *                  + sum_s X(x)_s ((1+gamma_mu) Y(x+mu))_s^dagger ]
 * with s the boundary sign of the hop.
 * Clover part: delta S = Re[c' sum_x sum_{mu<nu} tr(delta Q_{mu nu}(x) N)],
 * c' = -i kappa c_SW / 4, N = M + M^dagger,
 * M_ba = sum_{s,t} sigma_{mu nu}[s][t] X_{t b} conj(Y_{s a}).
 * For a leaf A_0 A_1 A_2 A_3 and the factor A_k, with
 * R_k = A_{k+1}..A_3 N A_0..A_{k-1}:  A_k = U gives g += conj(c') R_k^dagger,
 * A_k = U^dagger gives g += c' R_k.
 */
void or_force(const int *L, int tbc, double kappa, double csw, const cplx *U, const cplx *X,
              const cplx *Y, cplx *g)
{
    init_gamma();
    long V = vol4(L);
    for (long i = 0; i < V * 36; ++i) g[i] = 0;
    /* hopping part */
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu) {
            int crossed;
            long f = neighbour(x, mu, +1, L, &crossed);
            double sg = (mu == 3 && crossed) ? (double)tbc : 1.0;
            cplx A[4][3], B[4][3];
            for (int s = 0; s < 4; ++s)
                for (int a = 0; a < 3; ++a) {
                    cplx ga = 0, gb = 0;
                    for (int t = 0; t < 4; ++t) {
                        ga += G[mu][s][t] * Y[x * 12 + t * 3 + a];
                        gb += G[mu][s][t] * Y[f * 12 + t * 3 + a];
                    }
                    A[s][a] = Y[x * 12 + s * 3 + a] - ga;
                    B[s][a] = Y[f * 12 + s * 3 + a] + gb;
                }
            cplx *gl = g + (x * 4 + mu) * 9;
            for (int a = 0; a < 3; ++a)
                for (int bb = 0; bb < 3; ++bb) {
                    cplx acc = 0;
                    for (int s = 0; s < 4; ++s) {
                        acc += A[s][a] * conj(X[f * 12 + s * 3 + bb]);
                        acc += X[x * 12 + s * 3 + a] * conj(B[s][bb]);
                    }
                    gl[a * 3 + bb] += 2.0 * kappa * sg * acc;
                }
        }
    /* clover part */
    cplx cp = -I * kappa * csw / 4.0;
    for (long x = 0; x < V; ++x)
        for (int mu = 0; mu < 4; ++mu)
            for (int nu = mu + 1; nu < 4; ++nu) {
                cplx M[9], Md[9], N[9];
                for (int b = 0; b < 3; ++b)
                    for (int a = 0; a < 3; ++a) {
                        cplx acc = 0;
                        for (int s = 0; s < 4; ++s)
                            for (int t = 0; t < 4; ++t)
                                acc += SIG[mu][nu][s][t] * X[x * 12 + t * 3 + b] *
                                       conj(Y[x * 12 + s * 3 + a]);
                        M[b * 3 + a] = acc;
                    }
                m3_dag(M, Md);
                for (int i = 0; i < 9; ++i) N[i] = M[i] + Md[i];
                factor_t f[4][4];
                leaf_factors(x, mu, nu, L, f);
                for (int l = 0; l < 4; ++l)
                    for (int k = 0; k < 4; ++k) {
                        cplx R[9], A[9];
                        m3_identity(R);
                        for (int q = k + 1; q < 4; ++q) {
                            factor_matrix(U, f[l][q], A);
                            m3_mul(R, A, R);
                        }
                        m3_mul(R, N, R);
                        for (int q = 0; q < k; ++q) {
                            factor_matrix(U, f[l][q], A);
                            m3_mul(R, A, R);
                        }
                        cplx *gl = g + (f[l][k].site * 4 + f[l][k].dir) * 9;
                        if (f[l][k].dag) {
                            for (int i = 0; i < 9; ++i) gl[i] += cp * R[i];
                        } else {
                            cplx Rd[9];
                            m3_dag(R, Rd);
                            for (int i = 0; i < 9; ++i) gl[i] += conj(cp) * Rd[i];
                        }
                    }
            }
}
