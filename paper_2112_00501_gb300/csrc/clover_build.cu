// The clover term of Eq. (1) and its inverse, built on the GPU in FP64 from
// the gauge field (Sec. 2: C and C^-1 are computed from the gauge field).
//
//   F_{mu nu}(x) = (Q_{mu nu}(x) - Q_{mu nu}(x)^+) / 8,
//   Q_{mu nu}(x) = sum of the four plaquette leaves in the mu-nu plane that
//                  start and end at x (orientation mu then nu),
//   C = 1 + i kappa c_SW sum_{mu<nu} sigma_{mu nu} F_{mu nu}.
// In the chiral basis sigma_{mu nu} = diag(s+_{mu nu}, s-_{mu nu}) with 2x2
// blocks built from Pauli matrices (table below), so C = diag(C+, C-) with
// two 6x6 Hermitian blocks; each block is inverted by Gauss-Jordan
// elimination with partial pivoting.
#include "mgc_host.h"
#include "sigma.cuh"

namespace mgc {

typedef Cx<double> cd;

__device__ void m3mul(const cd *a, const cd *b, cd *o)
{
    cd t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) {
            cd acc = a[i * 3] * b[j];
            acc = cfma(a[i * 3 + 1], b[3 + j], acc);
            acc = cfma(a[i * 3 + 2], b[6 + j], acc);
            t[i * 3 + j] = acc;
        }
    for (int k = 0; k < 9; ++k) o[k] = t[k];
}

__device__ void m3dag(const cd *a, cd *o)
{
    cd t[9];
    for (int i = 0; i < 3; ++i)
        for (int j = 0; j < 3; ++j) t[i * 3 + j] = conj(a[j * 3 + i]);
    for (int k = 0; k < 9; ++k) o[k] = t[k];
}

__device__ int shifted_site(const Geom &g, const int c[4], int mu, int dm, int nu, int dn)
{
    int n[4] = {c[0], c[1], c[2], c[3]};
    n[mu] = (n[mu] + dm + g.L[mu]) % g.L[mu];
    n[nu] = (n[nu] + dn + g.L[nu]) % g.L[nu];
    return site_index(g, n);
}

// link U_dir(site), optionally daggered
__device__ void get_link(const Gauge64 &U, int site, int dir, bool dag, cd *o)
{
    U.load(site, dir, o);
    if (dag) m3dag(o, o);
}

// the sum of the four leaves of the mu-nu plane at site x (coordinates c)
__device__ void clover_leaves(const Geom &g, const Gauge64 &U, const int c[4], int x, int mu, int nu, cd *Q)
{
    const int xpm = shifted_site(g, c, mu, 1, nu, 0), xpn = shifted_site(g, c, mu, 0, nu, 1);
    const int xmm = shifted_site(g, c, mu, -1, nu, 0), xmn = shifted_site(g, c, mu, 0, nu, -1);
    const int xmmpn = shifted_site(g, c, mu, -1, nu, 1), xmmmn = shifted_site(g, c, mu, -1, nu, -1);
    const int xpmmn = shifted_site(g, c, mu, 1, nu, -1);
    cd P[9], A[9];
    for (int k = 0; k < 9; ++k) Q[k] = cd{0, 0};
    // U_mu(x) U_nu(x+mu) U_mu(x+nu)^+ U_nu(x)^+
    get_link(U, x, mu, false, P);
    get_link(U, xpm, nu, false, A); m3mul(P, A, P);
    get_link(U, xpn, mu, true, A); m3mul(P, A, P);
    get_link(U, x, nu, true, A); m3mul(P, A, P);
    for (int k = 0; k < 9; ++k) Q[k] = Q[k] + P[k];
    // U_nu(x) U_mu(x-mu+nu)^+ U_nu(x-mu)^+ U_mu(x-mu)
    get_link(U, x, nu, false, P);
    get_link(U, xmmpn, mu, true, A); m3mul(P, A, P);
    get_link(U, xmm, nu, true, A); m3mul(P, A, P);
    get_link(U, xmm, mu, false, A); m3mul(P, A, P);
    for (int k = 0; k < 9; ++k) Q[k] = Q[k] + P[k];
    // U_mu(x-mu)^+ U_nu(x-mu-nu)^+ U_mu(x-mu-nu) U_nu(x-nu)
    get_link(U, xmm, mu, true, P);
    get_link(U, xmmmn, nu, true, A); m3mul(P, A, P);
    get_link(U, xmmmn, mu, false, A); m3mul(P, A, P);
    get_link(U, xmn, nu, false, A); m3mul(P, A, P);
    for (int k = 0; k < 9; ++k) Q[k] = Q[k] + P[k];
    // U_nu(x-nu)^+ U_mu(x-nu) U_nu(x-nu+mu) U_mu(x)^+
    get_link(U, xmn, nu, true, P);
    get_link(U, xmn, mu, false, A); m3mul(P, A, P);
    get_link(U, xpmmn, nu, false, A); m3mul(P, A, P);
    get_link(U, x, mu, true, A); m3mul(P, A, P);
    for (int k = 0; k < 9; ++k) Q[k] = Q[k] + P[k];
}

// pack a Hermitian 6x6 (row-major) into 36 reals: diagonal, then lower triangle
__device__ void pack_herm6(const cd *A, double *out)
{
    for (int a = 0; a < 6; ++a) out[a] = A[a * 6 + a].r;
    int k = 6;
    for (int a = 1; a < 6; ++a)
        for (int b = 0; b < a; ++b) {
            out[k++] = A[a * 6 + b].r;
            out[k++] = A[a * 6 + b].i;
        }
}

// inverse of a 6x6 complex matrix, Gauss-Jordan with partial pivoting;
// returns false on an exactly zero pivot
__device__ bool invert6(const cd *A, cd *Ai)
{
    cd M[6][12];
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 12; ++j)
            M[i][j] = (j < 6) ? A[i * 6 + j] : cd{(j - 6 == i) ? 1.0 : 0.0, 0.0};
    for (int col = 0; col < 6; ++col) {
        int piv = col;
        double best = norm2(M[col][col]);
        for (int r = col + 1; r < 6; ++r)
            if (norm2(M[r][col]) > best) { best = norm2(M[r][col]); piv = r; }
        if (best == 0.0) return false;
        if (piv != col)
            for (int j = 0; j < 12; ++j) { cd t = M[col][j]; M[col][j] = M[piv][j]; M[piv][j] = t; }
        const cd d = M[col][col];
        const double dn = norm2(d);
        const cd inv = {d.r / dn, -d.i / dn};
        for (int j = 0; j < 12; ++j) M[col][j] = M[col][j] * inv;
        for (int r = 0; r < 6; ++r) {
            if (r == col) continue;
            const cd f = M[r][col];
            for (int j = 0; j < 12; ++j) M[r][j] = M[r][j] - f * M[col][j];
        }
    }
    for (int i = 0; i < 6; ++i)
        for (int j = 0; j < 6; ++j) Ai[i * 6 + j] = M[i][6 + j];
    return true;
}

__global__ void k_clover_build(Geom g, Gauge64 U, double kappa, double csw, double2 *C64, double2 *Ci64, int *bad)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    int c[4];
    site_coords(g, x, c);
    cd F[6][9];
    int p = 0;
    for (int mu = 0; mu < 4; ++mu)
        for (int nu = mu + 1; nu < 4; ++nu, ++p) {
            cd Q[9];
            clover_leaves(g, U, c, x, mu, nu, Q);
            for (int k = 0; k < 9; ++k) {
                const cd qd = conj(Q[(k % 3) * 3 + k / 3]);
                F[p][k] = 0.125 * (Q[k] - qd);
            }
        }
    const double kc = kappa * csw;
    const size_t base = ((size_t)(x >> g.lvb) * 36 << g.lvb) + (x & ((1 << g.lvb) - 1));
    for (int chi = 0; chi < 2; ++chi) {
        cd A[36], Ai[36];
        for (int s = 0; s < 2; ++s)
            for (int a = 0; a < 3; ++a)
                for (int t = 0; t < 2; ++t)
                    for (int b = 0; b < 3; ++b) {
                        cd acc = {(s == t && a == b) ? 1.0 : 0.0, 0.0};
                        for (int q = 0; q < 6; ++q) {
                            const cd sg = {c_sigma[chi][q][s][t][0], c_sigma[chi][q][s][t][1]};
                            // i kappa c_SW sigma F
                            const cd term = sg * F[q][a * 3 + b];
                            acc = acc + kc * times_i(term);
                        }
                        A[(s * 3 + a) * 6 + (t * 3 + b)] = acc;
                    }
        double pk[36];
        pack_herm6(A, pk);
        for (int k = 0; k < 18; ++k) C64[base + ((size_t)(chi * 18 + k) << g.lvb)] = make_double2(pk[2 * k], pk[2 * k + 1]);
        if (!invert6(A, Ai)) atomicAdd(bad, 1);
        pack_herm6(Ai, pk);
        for (int k = 0; k < 18; ++k) Ci64[base + ((size_t)(chi * 18 + k) << g.lvb)] = make_double2(pk[2 * k], pk[2 * k + 1]);
    }
}

int launch_clover_build(const Geom &g, const double2 *U64, double kappa, double csw, double2 *C64, double2 *Ci64,
                        int *d_bad, cudaStream_t s)
{
    k_clover_build<<<grid_for(g.V, 128), 128, 0, s>>>(g, Gauge64{(double2 *)U64, g.lvb}, kappa, csw, C64, Ci64, d_bad);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (576.0 + 2 * 576.0));
    return MGC_OK;
}

// FP64 packed clover -> FP32 (18 float4 planes) or FP16 (9 x 8 halves + scale)
__global__ void k_clover_lowprec(Geom g, Clover64 C, int prec, void *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    double c[72];
    C.load(x, c);
    const size_t l = x & ((1 << g.lvb) - 1), blk = x >> g.lvb;
    if (prec == 32) {
        float4 *o = (float4 *)out + (blk * 18 << g.lvb) + l;
        for (int k = 0; k < 18; ++k)
            o[(size_t)k << g.lvb] = make_float4((float)c[4 * k], (float)c[4 * k + 1], (float)c[4 * k + 2], (float)c[4 * k + 3]);
    } else {
        float m = 0.f;
        for (int k = 0; k < 72; ++k) m = fmaxf(m, fabsf((float)c[k]));
        const float inv = m > 0.f ? 1.0f / m : 0.f;
        uint4 *o = (uint4 *)out + (blk * 9 << g.lvb) + l;
        float *sc = (float *)((uint4 *)out + (size_t)g.V * 9);
        for (int k = 0; k < 9; ++k) {
            const double *q = c + 8 * k;
            o[(size_t)k << g.lvb] = make_uint4(pack_half2((float)q[0] * inv, (float)q[1] * inv),
                                               pack_half2((float)q[2] * inv, (float)q[3] * inv),
                                               pack_half2((float)q[4] * inv, (float)q[5] * inv),
                                               pack_half2((float)q[6] * inv, (float)q[7] * inv));
        }
        sc[x] = m;
    }
}

int launch_clover_lowprec(const Geom &g, const double2 *C64, int prec, void *out, cudaStream_t s)
{
    k_clover_lowprec<<<grid_for(g.V, 256), 256, 0, s>>>(g, Clover64{(double2 *)C64, g.lvb}, prec, out);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (576.0 + clover_site_bytes(prec)));
    return MGC_OK;
}

// packed FP64 clover -> canonical [s][12][12] complex128
__global__ void k_clover_export(Geom g, Clover64 C, double2 *out)
{
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    if (x >= g.V) return;
    int c[4];
    site_coords(g, x, c);
    double d[72];
    C.load(x, d);
    double2 *o = out + canon_index(g, c) * 144;
    for (int k = 0; k < 144; ++k) o[k] = make_double2(0.0, 0.0);
    for (int chi = 0; chi < 2; ++chi) {
        const double *q = d + 36 * chi;
        const int off = 6 * chi;
        for (int a = 0; a < 6; ++a) o[(off + a) * 12 + off + a] = make_double2(q[a], 0.0);
        int k = 6;
        for (int a = 1; a < 6; ++a)
            for (int b = 0; b < a; ++b) {
                o[(off + a) * 12 + off + b] = make_double2(q[k], q[k + 1]);
                o[(off + b) * 12 + off + a] = make_double2(q[k], -q[k + 1]);
                k += 2;
            }
    }
}

int launch_clover_export(const Geom &g, const double2 *C64, double *out, cudaStream_t s)
{
    k_clover_export<<<grid_for(g.V, 128), 128, 0, s>>>(g, Clover64{(double2 *)C64, g.lvb}, (double2 *)out);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (576.0 + 144 * 16.0));
    return MGC_OK;
}

// max over links of max|U U^+ - 1| and |det U - 1|, for 12-real compression
__global__ void k_unitarity(long long nlinks, const double2 *__restrict__ canon, unsigned long long *maxerr)
{
    const long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    double err = 0.0;
    if (n < nlinks) {
        cd u[9];
        for (int k = 0; k < 9; ++k) u[k] = cd{canon[n * 9 + k].x, canon[n * 9 + k].y};
        for (int i = 0; i < 3; ++i)
            for (int j = 0; j < 3; ++j) {
                cd acc = {0, 0};
                for (int k = 0; k < 3; ++k) acc = cfma(u[i * 3 + k], conj(u[j * 3 + k]), acc);
                if (i == j) acc.r -= 1.0;
                err = fmax(err, sqrt(norm2(acc)));
            }
        cd det = u[0] * (u[4] * u[8] - u[5] * u[7]) - u[1] * (u[3] * u[8] - u[5] * u[6]) +
                 u[2] * (u[3] * u[7] - u[4] * u[6]);
        det.r -= 1.0;
        err = fmax(err, sqrt(norm2(det)));
        if (!(err == err)) err = 1e300;  // NaN
    }
    // non-negative doubles order like their bit patterns
    atomicMax(maxerr, (unsigned long long)__double_as_longlong(err));
}

int launch_unitarity(const Geom &g, const double *canon_dev, double *d_maxerr, cudaStream_t s)
{
    const long long n = (long long)g.V * 4;
    k_unitarity<<<grid_for(n, 256), 256, 0, s>>>(n, (const double2 *)canon_dev, (unsigned long long *)d_maxerr);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)n * 144.0);
    return MGC_OK;
}

}  // namespace mgc
