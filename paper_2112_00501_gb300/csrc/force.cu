// Gauge-link force of S = phi^+ (D^+ D)^-1 phi (the HMC fermion force).
//
// With Y = D^-+ phi = gamma5 D^-1 gamma5 phi and X = D^-1 Y, a link variation
// gives delta S = -2 Re Y^+ (delta D) X, delta D = -kappa delta H + delta C.
// The returned tensor per link is g = dS/dRe U + i dS/dIm U, so that
// delta S = Re sum_ab conj(g_ab) delta U_ab.
//
//   hopping: g(x, mu) += 2 kappa s [ sum_s ((1 - gamma_mu) Y(x))_s X(x+mu)_s^+
//                                   + sum_s X(x)_s ((1 + gamma_mu) Y(x+mu))_s^+ ]
//            (s the t-boundary sign of the hop);
//   clover:  delta S = Re[c' sum_x sum_{mu<nu} tr(delta Q_{mu nu}(x) N_{mu nu}(x))],
//            c' = -i kappa c_SW / 4, N = M + M^+,
//            M_ba = sum_{s,t} sigma_{mu nu}[s][t] X_{t b}(x) conj(Y_{s a}(x)).
// Every plaquette of the mu-nu plane is a leaf of Q at each of its four
// corners.  For a link that appears undaggered in a plaquette the term is
// conj(c') R^+, daggered c' R, where R is the product of the plaquette's other
// three links M1 M2 M3 (in loop order after the link) with N(corner) inserted
// where the loop passes each corner:
//   R = N(c0) M1 M2 M3 + M1 N(c1) M2 M3 + M1 M2 N(c2) M3 + M1 M2 M3 N(c3).
#include <vector>

#include "hop.cuh"
#include "mgc_host.h"
#include "sigma.cuh"

namespace mgc {

typedef Cx<double> cd;

__device__ __forceinline__ void f_m3mul(const cd *a, const cd *b, cd *o)
{
    cd t[9];
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cd acc = a[i * 3] * b[j];
            acc = cfma(a[i * 3 + 1], b[3 + j], acc);
            acc = cfma(a[i * 3 + 2], b[6 + j], acc);
            t[i * 3 + j] = acc;
        }
#pragma unroll
    for (int k = 0; k < 9; ++k) o[k] = t[k];
}

// o += a b: the product's multiply-adds accumulate onto o (o distinct from a, b)
__device__ __forceinline__ void f_m3mul_acc(const cd *a, const cd *b, cd *o)
{
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) {
            cd acc = cfma(a[i * 3], b[j], o[i * 3 + j]);
            acc = cfma(a[i * 3 + 1], b[3 + j], acc);
            acc = cfma(a[i * 3 + 2], b[6 + j], acc);
            o[i * 3 + j] = acc;
        }
}

__device__ __forceinline__ void f_link(const Gauge64 &U, const Geom &g, const int c[4], int d0, int s0, int d1, int s1,
                                       int dir, bool dag, cd *o)
{
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[d0] = (n[d0] + s0 + g.L[d0]) % g.L[d0];
    n[d1] = (n[d1] + s1 + g.L[d1]) % g.L[d1];
    cd u[9];
    U.load(site_index(g, n), dir, u);
#pragma unroll
    for (int i = 0; i < 3; ++i)
#pragma unroll
        for (int j = 0; j < 3; ++j) o[i * 3 + j] = dag ? conj(u[j * 3 + i]) : u[i * 3 + j];
}

__device__ __forceinline__ void f_N(const double2 *N, const Geom &g, const int c[4], int d0, int s0, int d1, int s1,
                                    int plane, cd *o)
{
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[d0] = (n[d0] + s0 + g.L[d0]) % g.L[d0];
    n[d1] = (n[d1] + s1 + g.L[d1]) % g.L[d1];
    const double2 *q = N + ((size_t)site_index(g, n) * 6 + plane) * 9;
#pragma unroll
    for (int k = 0; k < 9; ++k) {
        double2 v = q[k];
        o[k] = cd{v.x, v.y};
    }
}

// N_{mu nu}(x) = M + M^+ for the six planes.  Each chiral block of sigma is
// a signed Pauli matrix: two of its four entries vanish and the others are
// +-1 or +-i, so with the loops unrolled over the constant table a nonzero
// entry costs the four multiply-adds of X_t conj(Y_s) into M and a zero one
// nothing.
__global__ void __launch_bounds__(128) k_force_N(Geom g, Spinor64 X, Spinor64 Y, double2 *N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    cd x[12], y[12];
    X.load(i, x);
    Y.load(i, y);
#pragma unroll
    for (int p = 0; p < 6; ++p) {
        cd M[9];
#pragma unroll
        for (int k = 0; k < 9; ++k) M[k] = cd{0, 0};
#pragma unroll
        for (int chi = 0; chi < 2; ++chi)
#pragma unroll
            for (int s = 0; s < 2; ++s)
#pragma unroll
                for (int t = 0; t < 2; ++t) {
                    const double sr = c_sigma[chi][p][s][t][0], si = c_sigma[chi][p][s][t][1];
                    if (sr == 0.0 && si == 0.0) continue;
#pragma unroll
                    for (int b = 0; b < 3; ++b)
#pragma unroll
                        for (int a = 0; a < 3; ++a) {
                            const cd xt = x[(2 * chi + t) * 3 + b], ys = y[(2 * chi + s) * 3 + a];
                            cd &m = M[b * 3 + a];
                            // m += sigma_st xt conj(ys), sigma_st = sr (real) or i si (imaginary)
                            if (si == 0.0) {
                                m.r = fma(sr * xt.r, ys.r, fma(sr * xt.i, ys.i, m.r));
                                m.i = fma(sr * xt.i, ys.r, fma(-sr * xt.r, ys.i, m.i));
                            } else {
                                m.r = fma(-si * xt.i, ys.r, fma(si * xt.r, ys.i, m.r));
                                m.i = fma(si * xt.r, ys.r, fma(si * xt.i, ys.i, m.i));
                            }
                        }
                }
        double2 *o = N + ((size_t)i * 6 + p) * 9;
#pragma unroll
        for (int r = 0; r < 3; ++r)
#pragma unroll
            for (int cc = 0; cc < 3; ++cc) {
                const cd v = M[r * 3 + cc] + conj(M[cc * 3 + r]);
                o[r * 3 + cc] = make_double2(v.r, v.i);
            }
    }
}


// The clover-leaf terms of all four links of one plaquette at once.  For the
// plaquette at x in the plane (mu, nu), mu < nu, with links in loop order
// A = U_mu(x), B = U_nu(x+mu), C = U_mu(x+nu)^+, D = U_nu(x)^+ and the
// insertions N0..N3 = N_{mu nu} at its corners x, x+mu, x+mu+nu, x+nu, the
// term of each link is the product of the other three in loop order after it
// with N inserted at each corner in turn (the R of the header).  With
// E_A = N0 A + A N1, E_B = N1 B + B N2, E_C = N2 C + C N3, E_D = N3 D + D N0:
//   R_A = E_B CD + BC E_D,  R_B = E_C DA + CD E_A,
//   R_C = E_D AB + DA E_B,  R_D = E_A BC + AB E_C.
// N is Hermitian, so a link's E in one plane is shared, daggered, by its two
// plaquettes there: with E_mu(x) = N(x) U_mu(x) + U_mu(x) N(x+mu) (k_force_E),
// E_A = E_mu(x), E_B = E_nu(x+mu), E_C = E_mu(x+nu)^+, E_D = E_nu(x)^+.
// 16 matrix products per plaquette for its four links (4 for the two E of
// each site and plane, 4 pair products, 8 for the R), against 32 when each
// link forms its own six terms.

// E_mu(x) and E_nu(x) of plane p (mu < nu), to Eb[((p * 2 + k) * 9 + e) * V + i]
// (k = 0: the link along mu, 1: along nu)
__global__ void __launch_bounds__(128) k_force_E(Geom g, Gauge64 U, const double2 *N, double2 *Eb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int p = blockIdx.y;
    const int mu = p < 3 ? 0 : (p < 5 ? 1 : 2);
    const int nu = p < 3 ? p + 1 : (p < 5 ? p - 1 : 3);
    int c[4];
    site_coords(g, i, c);
    const size_t V = (size_t)g.V;
#pragma unroll 1
    for (int k = 0; k < 2; ++k) {
        // the link from x along d = mu (k = 0) or nu (k = 1), N at both ends
        const int s0 = k == 0 ? 1 : 0, s1 = k == 0 ? 0 : 1;
        cd L[9], Nm[9], E[9];
        f_link(U, g, c, mu, 0, nu, 0, k == 0 ? mu : nu, false, L);
        f_N(N, g, c, mu, 0, nu, 0, p, Nm);
        f_m3mul(Nm, L, E);
        f_N(N, g, c, mu, s0, nu, s1, p, Nm);
        f_m3mul_acc(L, Nm, E);
        double2 *o = Eb + (size_t)(p * 2 + k) * 9 * V + i;
#pragma unroll
        for (int e = 0; e < 9; ++e) o[e * V] = make_double2(E[e].r, E[e].i);
    }
}

// R_A..R_D of the plaquette at x in plane p, to Rb[((p * 4 + X) * 9 + e) * V + i]
// (X = A, B, C, D as 0..3)
__global__ void __launch_bounds__(128) k_force_plaq(Geom g, Gauge64 U, const double2 *Eb, double2 *Rb)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int p = blockIdx.y;
    const int mu = p < 3 ? 0 : (p < 5 ? 1 : 2);
    const int nu = p < 3 ? p + 1 : (p < 5 ? p - 1 : 3);
    int c[4];
    site_coords(g, i, c);
    const size_t V = (size_t)g.V;
    auto put = [&](int X, const cd *R) {
        double2 *o = Rb + (size_t)(p * 4 + X) * 9 * V + i;
#pragma unroll
        for (int e = 0; e < 9; ++e) o[e * V] = make_double2(R[e].r, R[e].i);
    };
    // E of the link along mu (k = 0) or nu (k = 1) at x shifted by (s0, s1), daggered if dag
    auto getE = [&](int k, int s0, int s1, bool dag, cd *E) {
        int n[4] = {c[0], c[1], c[2], c[3]};
        n[mu] = (n[mu] + s0) % g.L[mu];
        n[nu] = (n[nu] + s1) % g.L[nu];
        const double2 *q = Eb + (size_t)(p * 2 + k) * 9 * V + site_index(g, n);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const double2 v = q[(dag ? b * 3 + a : a * 3 + b) * V];
                E[a * 3 + b] = dag ? cd{v.x, -v.y} : cd{v.x, v.y};
            }
    };
    // the four products of neighbouring links
    cd AB[9], BC[9], CD[9], DA[9];
    {
        cd X[9], Y[9];
        f_link(U, g, c, mu, 0, nu, 0, mu, false, X);  // A
        f_link(U, g, c, mu, 1, nu, 0, nu, false, Y);  // B
        f_m3mul(X, Y, AB);
        f_link(U, g, c, mu, 0, nu, 1, mu, true, X);   // C
        f_m3mul(Y, X, BC);
        f_link(U, g, c, mu, 0, nu, 0, nu, true, Y);   // D
        f_m3mul(X, Y, CD);
        f_link(U, g, c, mu, 0, nu, 0, mu, false, X);  // A
        f_m3mul(Y, X, DA);
    }
    // R = P Q + S T
    auto two = [&](const cd *P, const cd *Q, const cd *S, const cd *T, cd *R) {
        f_m3mul(P, Q, R);
        f_m3mul_acc(S, T, R);
    };
    cd E1[9], E2[9], R[9];
    getE(1, 1, 0, false, E1);  // E_B = E_nu(x+mu)
    getE(1, 0, 0, true, E2);   // E_D = E_nu(x)^+
    two(E1, CD, BC, E2, R);
    put(0, R);                 // R_A
    two(E2, AB, DA, E1, R);
    put(2, R);                 // R_C
    getE(0, 0, 0, false, E1);  // E_A = E_mu(x)
    getE(0, 0, 1, true, E2);   // E_C = E_mu(x+nu)^+
    two(E2, DA, CD, E1, R);
    put(1, R);                 // R_B
    two(E1, BC, AB, E2, R);
    put(3, R);                 // R_D
}

__device__ __forceinline__ int plane_of(int a, int b)
{
    // (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
}

// The hopping term of g(x, mu).  1 +- gamma_mu = R P with P the spin
// projection to a half spinor and R its reconstruction; the operator is
// Hermitian and its upper-left block the identity, so R = P^+ and
//   sum_s ((1 - gamma_mu) Y)_s conj(X_s) = sum_j (P Y)_j conj((P X)_j)
// over the two spins j of the half spinors: two projections and 18 complex
// products per term instead of a reconstruction and 36.
template <int MU>
__device__ void hop_force(const Geom &g, const int c[4], int i, const Spinor64 &X, const Spinor64 &Y, double kappa,
                          cd G[9])
{
    bool wr;
    const int f = neighbour(g, c, MU, +1, &wr);
    const double sg = (MU == 3 && wr && g.tbc < 0) ? -1.0 : 1.0;
    cd s[12], hy[6], hxf[6], hxx[6], hb[6];
    Y.load(i, s);
    project<MU, -1>(s, hy);   // P_- Y(x)
    X.load(f, s);
    project<MU, -1>(s, hxf);  // P_- X(x+mu)
    X.load(i, s);
    project<MU, +1>(s, hxx);  // P_+ X(x)
    Y.load(f, s);
    project<MU, +1>(s, hb);   // P_+ Y(x+mu)
    const double f2 = 2.0 * kappa * sg;
    // acc += u conj(v) as multiply-adds
    auto macc = [](cd &acc, cd u, cd v) {
        acc.r = fma(u.r, v.r, fma(u.i, v.i, acc.r));
        acc.i = fma(u.i, v.r, fma(-u.r, v.i, acc.i));
    };
#pragma unroll
    for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) {
            cd acc = {0, 0};
#pragma unroll
            for (int j = 0; j < 2; ++j) {
                macc(acc, hy[j * 3 + a], hxf[j * 3 + b]);
                macc(acc, hxx[j * 3 + a], hb[j * 3 + b]);
            }
            G[a * 3 + b] = cd{fma(f2, acc.r, G[a * 3 + b].r), fma(f2, acc.i, G[a * 3 + b].i)};
        }
}

// g(x, mu): the hopping term, then the clover-leaf terms of the six
// plaquettes that contain the link, read from k_force_plaq's output: in the
// plane (mu, s), s > mu, the link is A of the plaquette at x and C of the one
// at x - s; in the plane (s, mu), s < mu, it is B of the plaquette at x - s
// and D of the one at x.  Undaggered links take conj(c') R^+, daggered c' R.
__global__ void k_force(Geom g, Gauge64 U, Spinor64 X, Spinor64 Y, const double2 *Rb, double kappa, double csw,
                        double2 *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int mu = blockIdx.y;
    int c[4];
    site_coords(g, i, c);
    cd G[9];
    for (int k = 0; k < 9; ++k) G[k] = cd{0, 0};
    if (mu == 0) hop_force<0>(g, c, i, X, Y, kappa, G);
    else if (mu == 1) hop_force<1>(g, c, i, X, Y, kappa, G);
    else if (mu == 2) hop_force<2>(g, c, i, X, Y, kappa, G);
    else hop_force<3>(g, c, i, X, Y, kappa, G);

    // c' = -i kc with kc = kappa c_SW / 4: conj(c') R^+ adds kc (Im, Re) of
    // R's transpose, c' R adds kc (Im R, -Re R)
    const double kc = kappa * csw / 4.0;
    const size_t V = (size_t)g.V;
    auto get = [&](int p, int Xr, int site, cd *R) {
        const double2 *q = Rb + (size_t)(p * 4 + Xr) * 9 * V + site;
#pragma unroll
        for (int e = 0; e < 9; ++e) {
            const double2 v = q[e * V];
            R[e] = cd{v.x, v.y};
        }
    };
    for (int sgm = 0; sgm < 4; ++sgm) {
        if (sgm == mu) continue;
        const int p = plane_of(mu, sgm);
        int n[4] = {c[0], c[1], c[2], c[3]};
        n[sgm] = (n[sgm] - 1 + g.L[sgm]) % g.L[sgm];
        const int back = site_index(g, n);  // x - s
        cd R[9];
        // undaggered: A of the plaquette at x (mu < s) or B of the one at x - s (s < mu)
        if (mu < sgm) get(p, 0, i, R);
        else get(p, 1, back, R);
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                const cd r = R[b * 3 + a];
                G[a * 3 + b] = cd{fma(kc, r.i, G[a * 3 + b].r), fma(kc, r.r, G[a * 3 + b].i)};
            }
        // daggered: C of the plaquette at x - s (mu < s) or D of the one at x (s < mu)
        if (mu < sgm) get(p, 2, back, R);
        else get(p, 3, i, R);
#pragma unroll
        for (int k = 0; k < 9; ++k) G[k] = cd{fma(kc, R[k].i, G[k].r), fma(-kc, R[k].r, G[k].i)};
    }
    double2 *o = out + (canon_index(g, c) * 4 + mu) * 9;
    for (int k = 0; k < 9; ++k) o[k] = make_double2(G[k].r, G[k].i);
}

// S = 2 Re <phi, X> - ||D X||^2.  The two sums are nearly equal (both ~S), and
// central differences of S at small steps need S well beyond double precision
// (on 8^4, S ~ 5e4 has an ulp of 7e-12, which a step of 1e-5 turns into 4e-7
// of a derivative), so every product is split exactly into a double and its
// rounding error (fma), both are accumulated as unevaluated double-double
// pairs (Knuth's TwoSum), and the block partials are combined on the host the
// same way; S is returned as the pair (S rounded, remainder).
__device__ __forceinline__ void two_sum_acc(double &hi, double &lo, double v)
{
    const double s = hi + v;
    const double bp = s - hi;
    const double err = (hi - (s - bp)) + (v - bp);
    hi = s;
    lo += err;
}

// hi + lo += a * b, with the product's rounding error carried in lo
__device__ __forceinline__ void two_prod_acc(double &hi, double &lo, double a, double b)
{
    const double p = a * b;
    const double e = fma(a, b, -p);
    two_sum_acc(hi, lo, p);
    lo += e;
}

__global__ void k_action_partial(long long n, const double2 *phi, const double2 *X, const double2 *DX, double *part)
{
    __shared__ double sh[4][256];
    double ah = 0, al = 0, bh = 0, bl = 0;
    for (long long e = (long long)blockIdx.x * blockDim.x + threadIdx.x; e < n; e += (long long)gridDim.x * blockDim.x) {
        const double2 p = phi[e], x = X[e], d = DX[e];
        two_prod_acc(ah, al, p.x, x.x);
        two_prod_acc(ah, al, p.y, x.y);
        two_prod_acc(bh, bl, d.x, d.x);
        two_prod_acc(bh, bl, d.y, d.y);
    }
    sh[0][threadIdx.x] = ah;
    sh[1][threadIdx.x] = al;
    sh[2][threadIdx.x] = bh;
    sh[3][threadIdx.x] = bl;
    __syncthreads();
    for (int o = blockDim.x / 2; o > 0; o >>= 1) {
        if ((int)threadIdx.x < o) {
            double h = sh[0][threadIdx.x], l = sh[1][threadIdx.x] + sh[1][threadIdx.x + o];
            two_sum_acc(h, l, sh[0][threadIdx.x + o]);
            sh[0][threadIdx.x] = h;
            sh[1][threadIdx.x] = l;
            h = sh[2][threadIdx.x];
            l = sh[3][threadIdx.x] + sh[3][threadIdx.x + o];
            two_sum_acc(h, l, sh[2][threadIdx.x + o]);
            sh[2][threadIdx.x] = h;
            sh[3][threadIdx.x] = l;
        }
        __syncthreads();
    }
    if (threadIdx.x == 0)
        for (int k = 0; k < 4; ++k) part[4 * blockIdx.x + k] = sh[k][0];
}

static void host_two_sum(double &hi, double &lo, double v)
{
    const double s = hi + v;
    const double bp = s - hi;
    lo += (hi - (s - bp)) + (v - bp);
    hi = s;
}

int force(mgc_clover_s *op, const double *phi, double *dSdU, const mgc_solve_params *p, mgc_solve_info *info,
          double *action, cudaStream_t s)
{
    const Geom &g = op->gauge->lat->g;
    const size_t vb = spinor_bytes(g, 64, 1);
    const size_t gb = (size_t)g.V * 4 * 9 * sizeof(double2);
    double2 *phi64 = nullptr, *X = nullptr, *Y = nullptr, *T = nullptr, *N = nullptr, *stage = nullptr, *gout = nullptr;
    double2 *Rb = nullptr;  // the plaquettes' clover-leaf terms, 24 matrices per site
    double2 *Eb = nullptr;  // the links' N L + L N per plane, 12 matrices per site
    double *part = nullptr;
    int st = MGC_OK;
    mgc_solve_params q = *p;
    q.x_is_guess = 0;
    mgc_solve_info i1{}, i2{};
    const int nb = 512;
    auto cleanup = [&]() {
        cudaFree(phi64); cudaFree(X); cudaFree(Y); cudaFree(T); cudaFree(N); cudaFree(stage); cudaFree(gout);
        cudaFree(part); cudaFree(Rb); cudaFree(Eb);
    };
#define FTRY(call)                         \
    do {                                   \
        st = (call);                       \
        if (st != MGC_OK) { cleanup(); return st; } \
    } while (0)
#define FCUDA(call)                                                            \
    do {                                                                       \
        cudaError_t e_ = (call);                                               \
        if (e_ != cudaSuccess) { cleanup(); return cuda_fail(e_, #call, __FILE__, __LINE__); } \
    } while (0)
    FCUDA(cudaMalloc(&phi64, vb));
    FCUDA(cudaMalloc(&X, vb));
    FCUDA(cudaMalloc(&Y, vb));
    FCUDA(cudaMalloc(&T, vb));
    FCUDA(cudaMalloc(&N, (size_t)g.V * 54 * sizeof(double2)));
    FCUDA(cudaMalloc(&Rb, (size_t)g.V * 24 * 9 * sizeof(double2)));
    FCUDA(cudaMalloc(&Eb, (size_t)g.V * 12 * 9 * sizeof(double2)));
    FCUDA(cudaMalloc(&part, 4 * nb * sizeof(double)));
    if (!p->on_device) {
        FCUDA(cudaMalloc(&stage, vb));
        FCUDA(cudaMalloc(&gout, gb));
        FCUDA(cudaMemcpyAsync(stage, phi, vb, cudaMemcpyHostToDevice, s));
        FTRY(launch_pack(g, 64, 1, (const double *)stage, phi64, s));
    } else {
        FTRY(launch_pack(g, 64, 1, phi, phi64, s));
    }
    // Y = gamma5 D^-1 gamma5 phi
    FTRY(launch_gamma5(g, 1, phi64, T, s));
    st = solve_packed(op, T, Y, &q, &i1, s);
    if (st != MGC_OK) { *info = i1; cleanup(); return st; }
    FTRY(launch_gamma5(g, 1, Y, T, s));
    FCUDA(cudaMemcpyAsync(Y, T, vb, cudaMemcpyDeviceToDevice, s));
    // X = D^-1 Y
    st = solve_packed(op, Y, X, &q, &i2, s);
    if (st != MGC_OK) { *info = i2; cleanup(); return st; }
    info->status = MGC_OK;
    info->iters = i1.iters > i2.iters ? i1.iters : i2.iters;
    info->restarts = i1.restarts + i2.restarts;
    info->true_res = i1.true_res > i2.true_res ? i1.true_res : i2.true_res;
    if (action) {
        FTRY(launch_dirac(op, 64, false, X, T, 1, s));
        k_action_partial<<<nb, 256, 0, s>>>((long long)g.V * 12, phi64, X, T, part);
        FCUDA(cudaGetLastError());
        count(1, (double)g.V * 3 * 192.0);
        std::vector<double> h(4 * nb);
        FCUDA(cudaMemcpyAsync(h.data(), part, h.size() * sizeof(double), cudaMemcpyDeviceToHost, s));
        FCUDA(cudaStreamSynchronize(s));
        double ah = 0, al = 0, bh = 0, bl = 0;
        for (int k = 0; k < nb; ++k) {
            host_two_sum(ah, al, h[4 * k]);
            al += h[4 * k + 1];
            host_two_sum(bh, bl, h[4 * k + 2]);
            bl += h[4 * k + 3];
        }
        // 2a - b with the low parts carried along; action[0] + action[1] = S
        double sh = 0, sl = 0;
        host_two_sum(sh, sl, 2.0 * ah);
        host_two_sum(sh, sl, -bh);
        const double lo = sl + 2.0 * al - bl;
        action[0] = sh + lo;
        action[1] = lo - (action[0] - sh);
    }
    k_force_N<<<grid_for(g.V, 128), 128, 0, s>>>(g, Spinor64{X, g.lvb}, Spinor64{Y, g.lvb}, N);
    FCUDA(cudaGetLastError());
    count(1, (double)g.V * (2 * 192.0 + 54 * 16.0));
    k_force_E<<<dim3(grid_for(g.V, 128), 6), 128, 0, s>>>(g, Gauge64{op->gauge->U64, g.lvb}, N, Eb);
    FCUDA(cudaGetLastError());
    count(1, (double)g.V * (576.0 + 54 * 16.0 + 12 * 144.0));
    k_force_plaq<<<dim3(grid_for(g.V, 128), 6), 128, 0, s>>>(g, Gauge64{op->gauge->U64, g.lvb}, Eb, Rb);
    FCUDA(cudaGetLastError());
    count(1, (double)g.V * (576.0 + 12 * 144.0 + 24 * 144.0));
    double2 *dst = p->on_device ? (double2 *)dSdU : gout;
    dim3 grid(grid_for(g.V, 128), 4);
    k_force<<<grid, 128, 0, s>>>(g, Gauge64{op->gauge->U64, g.lvb}, Spinor64{X, g.lvb}, Spinor64{Y, g.lvb}, Rb,
                                 op->kappa, op->csw, dst);
    FCUDA(cudaGetLastError());
    count(1, (double)g.V * (2 * 192.0 + 24 * 144.0 + 576.0));
    if (!p->on_device) FCUDA(cudaMemcpyAsync(dSdU, gout, gb, cudaMemcpyDeviceToHost, s));
    FCUDA(cudaStreamSynchronize(s));
    cleanup();
#undef FTRY
#undef FCUDA
    return MGC_OK;
}

}  // namespace mgc
