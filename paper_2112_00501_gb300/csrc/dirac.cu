// Layout conversion and the fused clover-Wilson operator.
//
//  - pack / unpack / convert: canonical complex128 spinors <-> packed fields
//    at 64/32/16 bits, and packed <-> packed precision changes (the storage
//    conversions of the mixed-precision solver; FP16 carries one FP32 scale
//    per site).
//  - gauge pack: canonical links -> packed links (18 or 12 reals).
//  - k_dirac: out = C psi - kappa H psi (Eq. (1)), or D^dagger with the
//    projectors swapped, one thread per site; a right-hand-side index runs
//    over blockIdx.y.
//  - k_clover_apply: out = C psi or C^-1 psi.
#include "hop.cuh"
#include "hop16.cuh"
#include "mgc_host.h"

namespace mgc {

// ------------------------------------------------------------------ accessors
static Spinor64 sp64(const Geom &g, const void *b) { return Spinor64{(double2 *)b, g.lvb}; }
static Spinor32 sp32(const Geom &g, const void *b) { return Spinor32{(float4 *)b, g.lvb}; }
static Spinor16 sp16(const Geom &g, const void *b, int nrhs)
{
    uint4 *d = (uint4 *)b;
    return Spinor16{d, (float *)(d + (size_t)nrhs * g.V * 3), g.lvb};
}

size_t spinor_bytes(const Geom &g, int prec, int nrhs)
{
    const size_t V = (size_t)g.V * nrhs;
    if (prec == 64) return V * 192;
    if (prec == 32) return V * 96;
    return V * 48 + V * 4;
}

size_t gauge_bytes(const Geom &g, int prec, int compress)
{
    const size_t n = (size_t)g.V * 4;
    if (prec == 64) return n * 9 * 16;
    if (prec == 32) return compress == 12 ? n * 3 * 16 : n * 9 * 8;
    return compress == 12 ? n * 3 * 8 : n * 9 * 4;
}

size_t clover_bytes(const Geom &g, int prec)
{
    const size_t V = g.V;
    if (prec == 64) return V * 36 * 16;
    if (prec == 32) return V * 18 * 16;
    return V * 9 * 16 + V * 4;
}

// ------------------------------------------------------------------ pack
template <class SP>
__global__ void k_pack(Geom g, const double2 *__restrict__ canon, SP out)
{
    using T = typename SP::Real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    int c[4];
    site_coords(g, i, c);
    const double2 *q = canon + ((size_t)r * g.V + canon_index(g, c)) * 12;
    Cx<T> v[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) {
        double2 d = q[k];
        v[k] = Cx<T>{(T)d.x, (T)d.y};
    }
    shift_rhs(out, r, g.V).store(i, v);
}

template <class SP>
__global__ void k_unpack(Geom g, SP in, double2 *__restrict__ canon)
{
    using T = typename SP::Real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    int c[4];
    site_coords(g, i, c);
    Cx<T> v[12];
    shift_rhs(in, r, g.V).load(i, v);
    double2 *q = canon + ((size_t)r * g.V + canon_index(g, c)) * 12;
#pragma unroll
    for (int k = 0; k < 12; ++k) q[k] = make_double2((double)v[k].r, (double)v[k].i);
}

template <class SI, class SO>
__global__ void k_convert(Geom g, SI in, SO out)
{
    using TI = typename SI::Real;
    using TO = typename SO::Real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    Cx<TI> v[12];
    Cx<TO> w[12];
    shift_rhs(in, r, g.V).load(i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = Cx<TO>{(TO)v[k].r, (TO)v[k].i};
    shift_rhs(out, r, g.V).store(i, w);
}

int launch_pack(const Geom &g, int prec, int nrhs, const double *canon, void *packed, cudaStream_t s)
{
    dim3 grid(grid_for(g.V, 256), nrhs);
    const double2 *c = (const double2 *)canon;
    if (prec == 64) k_pack<<<grid, 256, 0, s>>>(g, c, sp64(g, packed));
    else if (prec == 32) k_pack<<<grid, 256, 0, s>>>(g, c, sp32(g, packed));
    else k_pack<<<grid, 256, 0, s>>>(g, c, sp16(g, packed, nrhs));
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * nrhs * (192.0 + spinor_site_bytes(prec)));
    return MGC_OK;
}

int launch_unpack(const Geom &g, int prec, int nrhs, const void *packed, double *canon, cudaStream_t s)
{
    dim3 grid(grid_for(g.V, 256), nrhs);
    double2 *c = (double2 *)canon;
    if (prec == 64) k_unpack<<<grid, 256, 0, s>>>(g, sp64(g, packed), c);
    else if (prec == 32) k_unpack<<<grid, 256, 0, s>>>(g, sp32(g, packed), c);
    else k_unpack<<<grid, 256, 0, s>>>(g, sp16(g, packed, nrhs), c);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * nrhs * (192.0 + spinor_site_bytes(prec)));
    return MGC_OK;
}

template <class SI>
static void convert_to(const Geom &g, int nrhs, SI in, int pout, void *out, cudaStream_t s)
{
    dim3 grid(grid_for(g.V, 256), nrhs);
    if (pout == 64) k_convert<<<grid, 256, 0, s>>>(g, in, sp64(g, out));
    else if (pout == 32) k_convert<<<grid, 256, 0, s>>>(g, in, sp32(g, out));
    else k_convert<<<grid, 256, 0, s>>>(g, in, sp16(g, out, nrhs));
}

int launch_convert(const Geom &g, int nrhs, int pin, const void *in, int pout, void *out, cudaStream_t s)
{
    if (pin == 64) convert_to(g, nrhs, sp64(g, in), pout, out, s);
    else if (pin == 32) convert_to(g, nrhs, sp32(g, in), pout, out, s);
    else convert_to(g, nrhs, sp16(g, in, nrhs), pout, out, s);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * nrhs * (spinor_site_bytes(pin) + spinor_site_bytes(pout)));
    return MGC_OK;
}

// ------------------------------------------------------------------ gauge pack
__global__ void k_gauge_pack(Geom g, const double2 *__restrict__ canon, int prec, int compress, void *out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int mu = blockIdx.y;
    int c[4];
    site_coords(g, i, c);
    const double2 *q = canon + (canon_index(g, c) * 4 + mu) * 9;
    const size_t l = i & ((1 << g.lvb) - 1);
    const size_t blk = i >> g.lvb;
    if (prec == 64) {
        double2 *o = (double2 *)out + ((blk * 4 + mu) * 9 << g.lvb) + l;
        for (int k = 0; k < 9; ++k) o[(size_t)k << g.lvb] = q[k];
    } else if (prec == 32 && compress == 18) {
        float2 *o = (float2 *)out + ((blk * 4 + mu) * 9 << g.lvb) + l;
        for (int k = 0; k < 9; ++k) o[(size_t)k << g.lvb] = make_float2((float)q[k].x, (float)q[k].y);
    } else if (prec == 32) {
        float4 *o = (float4 *)out + ((blk * 4 + mu) * 3 << g.lvb) + l;
        for (int k = 0; k < 3; ++k)
            o[(size_t)k << g.lvb] =
                make_float4((float)q[2 * k].x, (float)q[2 * k].y, (float)q[2 * k + 1].x, (float)q[2 * k + 1].y);
    } else if (compress == 18) {
        uint32_t *o = (uint32_t *)out + ((blk * 4 + mu) * 9 << g.lvb) + l;
        for (int k = 0; k < 9; ++k) o[(size_t)k << g.lvb] = pack_half2((float)q[k].x, (float)q[k].y);
    } else {
        uint2 *o = (uint2 *)out + ((blk * 4 + mu) * 3 << g.lvb) + l;
        for (int k = 0; k < 3; ++k)
            o[(size_t)k << g.lvb] = make_uint2(pack_half2((float)q[2 * k].x, (float)q[2 * k].y),
                                               pack_half2((float)q[2 * k + 1].x, (float)q[2 * k + 1].y));
    }
}

int launch_gauge_pack(const Geom &g, const double *canon_dev, int prec, int compress, void *out, cudaStream_t s)
{
    dim3 grid(grid_for(g.V, 256), 4);
    k_gauge_pack<<<grid, 256, 0, s>>>(g, (const double2 *)canon_dev, prec, compress, out);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (576.0 + links_site_bytes(prec, compress)));
    return MGC_OK;
}

// ------------------------------------------------------------------ D, D^dagger
// LVB > 0: cubic domains of 2^LVB sites, whose extents the compiler then knows
// (shifts and masks of the index arithmetic become constants); LVB == 0: any
// domain shape, read from g at run time.
// 128-thread blocks, five per SM for FP32 arithmetic (96 registers, no
// spills); measured against 256 x 2, 256 x 3 and 128 x 6 on 32^3 x 64.
constexpr int DIRAC_THREADS = 128;
// The input and output spinors may differ in storage (an FP16 input with the
// FP32 operator); the arithmetic type is theirs, which must agree.
template <bool DAG, int LVB, class SPI, class SPO, class GA, class CL>
__global__ void __launch_bounds__(DIRAC_THREADS, (LVB > 0 && sizeof(typename SPI::Real) == 4) ? 5 : 1)
    k_dirac(Geom g, SPI in, SPO out, GA U, CL C, typename SPI::Real kappa)
{
    using T = typename SPI::Real;
    static_assert(std::is_same<T, typename SPO::Real>::value, "input and output share the arithmetic type");
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    SPI src = shift_rhs(in, r, g.V);
    SPO dst = shift_rhs(out, r, g.V);
    GA Ug = U;
    CL Cg = C;
    Geom gg = g;
    if (LVB > 0) {
        gg.lvb = LVB;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LVB / 4;
        src.lvb = dst.lvb = Ug.lvb = Cg.lvb = LVB;
    }
    int c[4];
    site_coords(gg, i, c);
    if constexpr (sizeof(T) == 8) {
        const SPI one[1] = {src};
        Cx<T> o[1][12];
        dirac_site_pair<DAG, 1>(gg, c, i, one, 1, Ug, Cg, kappa, o);
        dst.store(i, o[0]);
    } else {
        Cx<T> o[12];
        dirac_site_k<DAG>(gg, c, i, src, Ug, Cg, kappa, o);
        dst.store(i, o);
    }
}

// ---- the FP16 operator: FP16 links, clover and spinors with their per-site
// scales, FP32 arithmetic with the FP16 factors fed to the multiply-adds as
// they are stored (hop16.cuh)

template <bool DAG, int LVB, class GA>
__global__ void __launch_bounds__(DIRAC_THREADS, 5)
    k_dirac16(Geom g, Spinor16 in, Spinor16 out, GA U, Clover16 C, float kappa)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    Spinor16 src = shift_rhs(in, r, g.V), dst = shift_rhs(out, r, g.V);
    GA Ug = U;
    Clover16 Cg = C;
    Geom gg = g;
    if (LVB > 0) {
        gg.lvb = LVB;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LVB / 4;
        src.lvb = dst.lvb = Ug.lvb = Cg.lvb = LVB;
    }
    int c[4];
    site_coords(gg, i, c);
    // C psi (with the clover and spinor scales), then the hops accumulated onto it
    float ar[12], ai[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) ar[k] = ai[k] = 0.f;
    {
        uint32_t v[12];
        words16(src, i, v);
        clover16_site(Cg, i, v, __ldg(Cg.sc + i) * src.scale_of(i), ar, ai);
    }
    hop16_dir<0, DAG>(gg, c, i, src, Ug, -kappa, ar, ai);
    hop16_dir<1, DAG>(gg, c, i, src, Ug, -kappa, ar, ai);
    hop16_dir<2, DAG>(gg, c, i, src, Ug, -kappa, ar, ai);
    hop16_dir<3, DAG>(gg, c, i, src, Ug, -kappa, ar, ai);
    Cx<float> o[12];
#pragma unroll
    for (int k = 0; k < 12; ++k) o[k] = Cx<float>{ar[k], ai[k]};
    dst.store(i, o);
}

template <int LVB, class GA>
static void dirac16_launch(const Geom &g, bool dag, Spinor16 in, Spinor16 out, GA U, Clover16 C, double kappa,
                           int nrhs, cudaStream_t s)
{
    dim3 grid(grid_for(g.V, DIRAC_THREADS), nrhs);
    if (dag) k_dirac16<true, LVB><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, C, (float)kappa);
    else k_dirac16<false, LVB><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, C, (float)kappa);
}

template <class GA>
static void dirac16_dispatch(const Geom &g, bool dag, Spinor16 in, Spinor16 out, GA U, Clover16 C, double kappa,
                             int nrhs, cudaStream_t s)
{
    const bool cube = g.lb[0] == g.lb[1] && g.lb[1] == g.lb[2] && g.lb[2] == g.lb[3];
    if (cube && g.lvb == 8) dirac16_launch<8>(g, dag, in, out, U, C, kappa, nrhs, s);
    else if (cube && g.lvb == 4) dirac16_launch<4>(g, dag, in, out, U, C, kappa, nrhs, s);
    else dirac16_launch<0>(g, dag, in, out, U, C, kappa, nrhs, s);
}

template <int LVB, class SPI, class SPO, class GA, class CL>
static void dirac_launch(const Geom &g, bool dag, SPI in, SPO out, GA U, CL C, double kappa, int nrhs, cudaStream_t s)
{
    using T = typename SPI::Real;
    dim3 grid(grid_for(g.V, DIRAC_THREADS), nrhs);
    if (dag) k_dirac<true, LVB><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, C, (T)kappa);
    else k_dirac<false, LVB><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, C, (T)kappa);
}

template <class SPI, class SPO, class GA, class CL>
static void dirac_dispatch(const Geom &g, bool dag, SPI in, SPO out, GA U, CL C, double kappa, int nrhs,
                           cudaStream_t s)
{
    const bool cube = g.lb[0] == g.lb[1] && g.lb[1] == g.lb[2] && g.lb[2] == g.lb[3];
    if (cube && g.lvb == 8) dirac_launch<8>(g, dag, in, out, U, C, kappa, nrhs, s);
    else if (cube && g.lvb == 4) dirac_launch<4>(g, dag, in, out, U, C, kappa, nrhs, s);
    else dirac_launch<0>(g, dag, in, out, U, C, kappa, nrhs, s);
}

static Clover16 cl16(const Geom &g, const mgc_clover_s *op)
{
    return Clover16{(uint4 *)op->C16, op->C16_sc, g.lvb};
}

int launch_dirac(const mgc_clover_s *op, int prec, bool dag, const void *in, void *out, int nrhs, cudaStream_t s)
{
    const mgc_gauge_s *ga = op->gauge;
    const Geom &g = ga->lat->g;
    if (!has_prec(ga, prec)) return fail(MGC_ERR_INVALID_ARG, "no copy of the operator at this precision");
    if (prec == 64) {
        dirac_dispatch(g, dag, sp64(g, in), sp64(g, out), Gauge64{ga->U64, g.lvb}, Clover64{op->C64, g.lvb},
                       op->kappa, nrhs, s);
    } else if (prec == 32) {
        Clover32 C{(float4 *)op->C32, g.lvb};
        if (ga->compress == 12)
            dirac_dispatch(g, dag, sp32(g, in), sp32(g, out), Gauge32x12{(float4 *)ga->U32, g.lvb}, C, op->kappa,
                           nrhs, s);
        else
            dirac_dispatch(g, dag, sp32(g, in), sp32(g, out), Gauge32x18{(float2 *)ga->U32, g.lvb}, C, op->kappa,
                           nrhs, s);
    } else {
        if (ga->compress == 12)
            dirac16_dispatch(g, dag, sp16(g, in, nrhs), sp16(g, out, nrhs), Gauge16x12{(uint2 *)ga->U16, g.lvb},
                             cl16(g, op), op->kappa, nrhs, s);
        else
            dirac16_dispatch(g, dag, sp16(g, in, nrhs), sp16(g, out, nrhs), Gauge16x18{(uint32_t *)ga->U16, g.lvb},
                             cl16(g, op), op->kappa, nrhs, s);
    }
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (2.0 * nrhs * spinor_site_bytes(prec) +
                            links_site_bytes(prec, prec == 64 ? 18 : ga->compress) + clover_site_bytes(prec)));
    return MGC_OK;
}

// w = D z for an FP16 z (per-site scale) with the FP32 operator: FP32
// arithmetic and result, the FP16 input read directly (the smoother's output
// in the mixed-precision solve, with no FP32 copy of it)
int launch_dirac_from16(const mgc_clover_s *op, const void *in16, void *out32, cudaStream_t s)
{
    const mgc_gauge_s *ga = op->gauge;
    const Geom &g = ga->lat->g;
    if (!has_prec(ga, 32)) return fail(MGC_ERR_INVALID_ARG, "no FP32 copy of the operator");
    Clover32 C{(float4 *)op->C32, g.lvb};
    if (ga->compress == 12)
        dirac_dispatch(g, false, sp16(g, in16, 1), sp32(g, out32), Gauge32x12{(float4 *)ga->U32, g.lvb}, C,
                       op->kappa, 1, s);
    else
        dirac_dispatch(g, false, sp16(g, in16, 1), sp32(g, out32), Gauge32x18{(float2 *)ga->U32, g.lvb}, C,
                       op->kappa, 1, s);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (spinor_site_bytes(16) + spinor_site_bytes(32) + links_site_bytes(32, ga->compress) +
                            clover_site_bytes(32)));
    return MGC_OK;
}

// ------------------------------------------------------------------ A = C^-1 D
// QWS's clover-preconditioned operator (Sec. 2): A psi = psi - kappa C^-1 H psi,
// one thread per site, the same hopping sum as k_dirac followed by C^-1, in
// k_dirac's launch shape.
template <int LVB, class SP, class GA, class CL>
__global__ void __launch_bounds__(DIRAC_THREADS, (LVB > 0 && sizeof(typename SP::Real) == 4) ? 5 : 1)
    k_apply_A(Geom g, SP in, SP out, GA U, CL Ci, typename SP::Real kappa)
{
    using T = typename SP::Real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    SP src = shift_rhs(in, r, g.V), dst = shift_rhs(out, r, g.V);
    GA Ug = U;
    CL Cg = Ci;
    Geom gg = g;
    if (LVB > 0) {
        gg.lvb = LVB;
#pragma unroll
        for (int mu = 0; mu < 4; ++mu) gg.lb[mu] = LVB / 4;
        src.lvb = dst.lvb = Ug.lvb = Cg.lvb = LVB;
    }
    int c[4];
    site_coords(gg, i, c);
    Cx<T> acc[12], t[12], psi[12];
    hop_site<false>(gg, c, i, src, Ug, acc);
    clover_site(Cg, i, acc, t);
    src.load(i, psi);
#pragma unroll
    for (int k = 0; k < 12; ++k) psi[k] = Cx<T>{fma(-kappa, t[k].r, psi[k].r), fma(-kappa, t[k].i, psi[k].i)};
    dst.store(i, psi);
}

template <class SP, class GA, class CL>
static void apply_A_dispatch(const Geom &g, SP in, SP out, GA U, CL Ci, double kappa, int nrhs, cudaStream_t s)
{
    using T = typename SP::Real;
    const bool cube = g.lb[0] == g.lb[1] && g.lb[1] == g.lb[2] && g.lb[2] == g.lb[3];
    dim3 grid(grid_for(g.V, DIRAC_THREADS), nrhs);
    if (cube && g.lvb == 8) k_apply_A<8><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, Ci, (T)kappa);
    else if (cube && g.lvb == 4) k_apply_A<4><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, Ci, (T)kappa);
    else k_apply_A<0><<<grid, DIRAC_THREADS, 0, s>>>(g, in, out, U, Ci, (T)kappa);
}

int launch_apply_A(const mgc_clover_s *op, int prec, const void *in, void *out, int nrhs, cudaStream_t s)
{
    const mgc_gauge_s *ga = op->gauge;
    const Geom &g = ga->lat->g;
    if (!has_prec(ga, prec)) return fail(MGC_ERR_INVALID_ARG, "no copy of the operator at this precision");
    if (prec == 64) {
        apply_A_dispatch(g, sp64(g, in), sp64(g, out), Gauge64{ga->U64, g.lvb}, Clover64{op->Ci64, g.lvb}, op->kappa,
                         nrhs, s);
    } else if (prec == 32) {
        Clover32 Ci{(float4 *)op->Ci32, g.lvb};
        if (ga->compress == 12)
            apply_A_dispatch(g, sp32(g, in), sp32(g, out), Gauge32x12{(float4 *)ga->U32, g.lvb}, Ci, op->kappa, nrhs,
                             s);
        else
            apply_A_dispatch(g, sp32(g, in), sp32(g, out), Gauge32x18{(float2 *)ga->U32, g.lvb}, Ci, op->kappa, nrhs,
                             s);
    } else {
        Clover16 Ci{(uint4 *)op->Ci16, op->Ci16_sc, g.lvb};
        if (ga->compress == 12)
            apply_A_dispatch(g, sp16(g, in, nrhs), sp16(g, out, nrhs), Gauge16x12{(uint2 *)ga->U16, g.lvb}, Ci,
                             op->kappa, nrhs, s);
        else
            apply_A_dispatch(g, sp16(g, in, nrhs), sp16(g, out, nrhs), Gauge16x18{(uint32_t *)ga->U16, g.lvb}, Ci,
                             op->kappa, nrhs, s);
    }
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (2.0 * nrhs * spinor_site_bytes(prec) +
                            links_site_bytes(prec, prec == 64 ? 18 : ga->compress) + clover_site_bytes(prec)));
    return MGC_OK;
}

// ------------------------------------------------------------------ clover apply
template <class SP, class CL>
__global__ void k_clover_apply(Geom g, SP in, SP out, CL C)
{
    using T = typename SP::Real;
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    Cx<T> v[12], o[12];
    shift_rhs(in, r, g.V).load(i, v);
    T cl[72];
    C.load(i, cl);
    clover_mul(cl, v, o);
    shift_rhs(out, r, g.V).store(i, o);
}

int launch_clover_apply(const mgc_clover_s *op, int prec, bool inverse, const void *in, void *out, int nrhs,
                        cudaStream_t s)
{
    const Geom &g = op->gauge->lat->g;
    dim3 grid(grid_for(g.V, 256), nrhs);
    if (prec == 64) {
        k_clover_apply<<<grid, 256, 0, s>>>(g, sp64(g, in), sp64(g, out),
                                            Clover64{inverse ? op->Ci64 : op->C64, g.lvb});
    } else if (!has_prec(op->gauge, prec)) {
        return fail(MGC_ERR_INVALID_ARG, "no copy of the clover term at this precision");
    } else if (prec == 32) {
        k_clover_apply<<<grid, 256, 0, s>>>(g, sp32(g, in), sp32(g, out),
                                            Clover32{(float4 *)(inverse ? op->Ci32 : op->C32), g.lvb});
    } else {
        const Clover16 C = inverse ? Clover16{(uint4 *)op->Ci16, op->Ci16_sc, g.lvb} : cl16(g, op);
        k_clover_apply<<<grid, 256, 0, s>>>(g, sp16(g, in, nrhs), sp16(g, out, nrhs), C);
    }
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (2.0 * nrhs * spinor_site_bytes(prec) + clover_site_bytes(prec)));
    return MGC_OK;
}

// ------------------------------------------------------------------ mixed-precision site kernels
// out32 = s * in64 (rounded to nearest) and x64 += c * e32, site by site so
// that the two packed layouts line up component by component
__global__ void k_scale_to32(Geom g, Spinor64 in, Spinor32 out, double s)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    Cx<double> v[12];
    Cx<float> w[12];
    in.load(i, v);
#pragma unroll
    for (int k = 0; k < 12; ++k) w[k] = Cx<float>{(float)(s * v[k].r), (float)(s * v[k].i)};
    out.store(i, w);
}

__global__ void k_axpy_from32(Geom g, Spinor64 x, Spinor32 e, double cr, double ci)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    Cx<double> v[12];
    Cx<float> d[12];
    x.load(i, v);
    e.load(i, d);
    const Cx<double> c = {cr, ci};
#pragma unroll
    for (int k = 0; k < 12; ++k) v[k] = cfma(c, Cx<double>{(double)d[k].r, (double)d[k].i}, v[k]);
    x.store(i, v);
}

int launch_scale_to32(const Geom &g, const double2 *in, void *out, double s, cudaStream_t st)
{
    k_scale_to32<<<grid_for(g.V, 256), 256, 0, st>>>(g, sp64(g, in), sp32(g, out), s);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (192.0 + 96.0));
    return MGC_OK;
}

int launch_axpy_from32(const Geom &g, double2 *x, const void *e, double cr, double ci, cudaStream_t st)
{
    k_axpy_from32<<<grid_for(g.V, 256), 256, 0, st>>>(g, sp64(g, x), sp32(g, e), cr, ci);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * (2 * 192.0 + 96.0));
    return MGC_OK;
}

// ------------------------------------------------------------------ gamma5
__global__ void k_gamma5(Geom g, int nrhs, const double2 *__restrict__ in, double2 *__restrict__ out)
{
    const int i = blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= g.V) return;
    const int r = blockIdx.y;
    Spinor64 a = shift_rhs(Spinor64{(double2 *)in, g.lvb}, r, g.V);
    Spinor64 b = shift_rhs(Spinor64{out, g.lvb}, r, g.V);
    Cx<double> v[12];
    a.load(i, v);
#pragma unroll
    for (int k = 6; k < 12; ++k) v[k] = -v[k];
    b.store(i, v);
}

int launch_gamma5(const Geom &g, int nrhs, const double2 *in, double2 *out, cudaStream_t s)
{
    dim3 grid(grid_for(g.V, 256), nrhs);
    k_gamma5<<<grid, 256, 0, s>>>(g, nrhs, in, out);
    MGC_CUDA(cudaGetLastError());
    count(1, (double)g.V * nrhs * 384.0);
    return MGC_OK;
}

}  // namespace mgc
