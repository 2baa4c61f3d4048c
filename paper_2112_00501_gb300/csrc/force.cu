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

// N_{mu nu}(x) = M + M^+ for the six planes
__global__ void k_force_N(Geom g, Spinor64 X, Spinor64 Y, double2 *N)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    cd x[12], y[12];
    X.load(i, x);
    Y.load(i, y);
    for (int p = 0; p < 6; ++p) {
        cd M[9];
        for (int b = 0; b < 3; ++b)
            for (int a = 0; a < 3; ++a) {
                cd acc = {0, 0};
                for (int chi = 0; chi < 2; ++chi)
                    for (int s = 0; s < 2; ++s)
                        for (int t = 0; t < 2; ++t) {
                            const cd sg = {c_sigma[chi][p][s][t][0], c_sigma[chi][p][s][t][1]};
                            const cd xt = x[(2 * chi + t) * 3 + b];
                            const cd ys = y[(2 * chi + s) * 3 + a];
                            acc = acc + sg * (xt * conj(ys));
                        }
                M[b * 3 + a] = acc;
            }
        double2 *o = N + ((size_t)i * 6 + p) * 9;
        for (int r = 0; r < 3; ++r)
            for (int cc = 0; cc < 3; ++cc) {
                const cd v = M[r * 3 + cc] + conj(M[cc * 3 + r]);
                o[r * 3 + cc] = make_double2(v.r, v.i);
            }
    }
}


// where a factor of a plaquette term sits relative to site c: a link
// (shifts along d0, d1; its direction; daggered or not) or an insertion N
struct LinkRef {
    int d0, s0, d1, s1, dir;
    bool dag;
};
struct NRef {
    int d0, s0, d1, s1;
};

// R = N0 M1 M2 M3 + M1 N1 M2 M3 + M1 M2 N2 M3 + M1 M2 M3 N3 with shared
// prefixes, each factor loaded just before its product, so that four 3x3
// matrices are live at a time (preloading all seven factors made the kernel
// spill)
__device__ void corner_sum(const Gauge64 &U, const double2 *N, const Geom &g, const int c[4], int p,
                                const LinkRef m[3], const NRef n[4], cd *R)
{
    cd A[9], B[9], T[9], P[9];
    f_link(U, g, c, m[0].d0, m[0].s0, m[0].d1, m[0].s1, m[0].dir, m[0].dag, A);  // M1
    f_N(N, g, c, n[0].d0, n[0].s0, n[0].d1, n[0].s1, p, B);
    f_m3mul(B, A, T);  // N0 M1
    f_N(N, g, c, n[1].d0, n[1].s0, n[1].d1, n[1].s1, p, B);
    f_m3mul(A, B, P);
    for (int k = 0; k < 9; ++k) T[k] = T[k] + P[k];  // N0 M1 + M1 N1
    f_link(U, g, c, m[1].d0, m[1].s0, m[1].d1, m[1].s1, m[1].dir, m[1].dag, B);  // M2
    f_m3mul(A, B, P);  // M1 M2
    f_m3mul(T, B, A);  // (..) M2
    f_N(N, g, c, n[2].d0, n[2].s0, n[2].d1, n[2].s1, p, B);
    f_m3mul(P, B, T);
    for (int k = 0; k < 9; ++k) T[k] = A[k] + T[k];  // (..) M2 + M1 M2 N2
    f_link(U, g, c, m[2].d0, m[2].s0, m[2].d1, m[2].s1, m[2].dir, m[2].dag, B);  // M3
    f_m3mul(P, B, A);  // M1 M2 M3
    f_m3mul(T, B, P);  // (..) M3
    f_N(N, g, c, n[3].d0, n[3].s0, n[3].d1, n[3].s1, p, B);
    f_m3mul(A, B, T);  // M1 M2 M3 N3
    for (int k = 0; k < 9; ++k) R[k] = P[k] + T[k];
}

__device__ __forceinline__ int plane_of(int a, int b)
{
    // (0,1) (0,2) (0,3) (1,2) (1,3) (2,3)
    const int lo = a < b ? a : b, hi = a < b ? b : a;
    return lo == 0 ? hi - 1 : (lo == 1 ? hi + 1 : 5);
}

template <int MU>
__device__ void hop_force(const Geom &g, const int c[4], int i, const Spinor64 &X, const Spinor64 &Y, double kappa,
                          cd G[9])
{
    bool wr;
    const int f = neighbour(g, c, MU, +1, &wr);
    const double sg = (MU == 3 && wr && g.tbc < 0) ? -1.0 : 1.0;
    cd yx[12], yf[12], xx[12], xf[12], h[6], A[12], B[12];
    Y.load(i, yx);
    Y.load(f, yf);
    X.load(i, xx);
    X.load(f, xf);
    for (int k = 0; k < 12; ++k) A[k] = B[k] = cd{0, 0};
    project<MU, -1>(yx, h);
    reconstruct_add<MU, -1>(A, h);  // (1 - gamma_mu) Y(x)
    project<MU, +1>(yf, h);
    reconstruct_add<MU, +1>(B, h);  // (1 + gamma_mu) Y(x+mu)
    const double f2 = 2.0 * kappa * sg;
    for (int a = 0; a < 3; ++a)
        for (int b = 0; b < 3; ++b) {
            cd acc = {0, 0};
            for (int s = 0; s < 4; ++s) {
                acc = acc + A[s * 3 + a] * conj(xf[s * 3 + b]);
                acc = acc + xx[s * 3 + a] * conj(B[s * 3 + b]);
            }
            G[a * 3 + b] = G[a * 3 + b] + f2 * acc;
        }
}

__global__ void k_force(Geom g, Gauge64 U, Spinor64 X, Spinor64 Y, const double2 *N, double kappa, double csw,
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

    const cd cp = {0.0, -kappa * csw / 4.0};  // c'
    const cd cpc = conj(cp);
    for (int sgm = 0; sgm < 4; ++sgm) {
        if (sgm == mu) continue;
        const int p = plane_of(mu, sgm);
        cd R[9];
        // undaggered plaquette
        if (mu < sgm) {
            // U_mu(y) U_s(y+mu) U_mu(y+s)^+ U_s(y)^+
            const LinkRef m[3] = {{mu, 1, sgm, 0, sgm, false}, {mu, 0, sgm, 1, mu, true}, {mu, 0, sgm, 0, sgm, true}};
            const NRef n[4] = {{mu, 1, sgm, 0}, {mu, 1, sgm, 1}, {mu, 0, sgm, 1}, {mu, 0, sgm, 0}};
            corner_sum(U, N, g, c, p, m, n, R);
        } else {
            // U_s(y-s) U_mu(y) U_s(y-s+mu)^+ U_mu(y-s)^+
            const LinkRef m[3] = {{sgm, -1, mu, 1, sgm, true}, {sgm, -1, mu, 0, mu, true}, {sgm, -1, mu, 0, sgm, false}};
            const NRef n[4] = {{sgm, 0, mu, 1}, {sgm, -1, mu, 1}, {sgm, -1, mu, 0}, {sgm, 0, mu, 0}};
            corner_sum(U, N, g, c, p, m, n, R);
        }
        for (int a = 0; a < 3; ++a)
            for (int b = 0; b < 3; ++b) G[a * 3 + b] = G[a * 3 + b] + cpc * conj(R[b * 3 + a]);
        // daggered plaquette
        if (mu < sgm) {
            // U_mu(y-s) U_s(y-s+mu) U_mu(y)^+ U_s(y-s)^+ ; after the link: y -> y-s -> y-s+mu -> y+mu
            const LinkRef m[3] = {{mu, 0, sgm, -1, sgm, true}, {mu, 0, sgm, -1, mu, false}, {mu, 1, sgm, -1, sgm, false}};
            const NRef n[4] = {{mu, 0, sgm, 0}, {mu, 0, sgm, -1}, {mu, 1, sgm, -1}, {mu, 1, sgm, 0}};
            corner_sum(U, N, g, c, p, m, n, R);
        } else {
            // U_s(y) U_mu(y+s) U_s(y+mu)^+ U_mu(y)^+ ; after the link: y -> y+s -> y+s+mu -> y+mu
            const LinkRef m[3] = {{sgm, 0, mu, 0, sgm, false}, {sgm, 1, mu, 0, mu, false}, {sgm, 0, mu, 1, sgm, true}};
            const NRef n[4] = {{sgm, 0, mu, 0}, {sgm, 1, mu, 0}, {sgm, 1, mu, 1}, {sgm, 0, mu, 1}};
            corner_sum(U, N, g, c, p, m, n, R);
        }
        for (int k = 0; k < 9; ++k) G[k] = G[k] + cp * R[k];
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
    double *part = nullptr;
    int st = MGC_OK;
    mgc_solve_params q = *p;
    q.x_is_guess = 0;
    mgc_solve_info i1{}, i2{};
    const int nb = 512;
    auto cleanup = [&]() {
        cudaFree(phi64); cudaFree(X); cudaFree(Y); cudaFree(T); cudaFree(N); cudaFree(stage); cudaFree(gout);
        cudaFree(part);
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
    double2 *dst = p->on_device ? (double2 *)dSdU : gout;
    dim3 grid(grid_for(g.V, 128), 4);
    k_force<<<grid, 128, 0, s>>>(g, Gauge64{op->gauge->U64, g.lvb}, Spinor64{X, g.lvb}, Spinor64{Y, g.lvb}, N,
                                 op->kappa, op->csw, dst);
    FCUDA(cudaGetLastError());
    count(1, (double)g.V * (2 * 192.0 + 54 * 16.0 + 576.0 + 576.0));
    if (!p->on_device) FCUDA(cudaMemcpyAsync(dSdU, gout, gb, cudaMemcpyDeviceToHost, s));
    FCUDA(cudaStreamSynchronize(s));
    cleanup();
#undef FTRY
#undef FCUDA
    return MGC_OK;
}

}  // namespace mgc
