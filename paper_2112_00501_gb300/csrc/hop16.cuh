// FP32 arithmetic on FP16-stored operands, for the fields kept in FP16 with a
// per-site scale (links, clover term, spinors): every product takes its two
// factors straight from the stored halves with the mixed-precision fused
// multiply-add of sm_100 and later (fma.rn.f32.f16: two FP16 factors, FP32
// addend and result).  The product of two FP16 numbers is exact in FP32, so
// each term is what FP32 arithmetic on the converted halves would give, and no
// FP16-to-FP32 conversion instruction is spent; the GB300 issues this FMA at
// the FP32 FMA rate.  The per-site scales, -kappa and the boundary sign enter
// once per hop as the real coefficient of the FP32 accumulation.
//
// A complex number is one 32-bit word: the real part in the low half, the
// imaginary part in the high half; a complex product is four FMAs on the
// halves.
//
// The spin projection of the hopping term (Eq. (1)) is formed on the packed
// halves (one FP16 addition per component), so the projected half spinor, the
// FP16 factor of the link products, carries one more FP16 rounding than the
// stored spinor.
#pragma once

#include <cuda_fp16.h>

#include "mgc_device.cuh"

namespace mgc {

// The products below split each 32-bit word into its halves inside one asm
// block (mov.b32 {lo, hi}), which addresses the halves in place, and negate a
// factor there (folded into the multiply-add): no instruction is spent on
// extracting, swapping or negating halves.

// acc += u * h:  re += u.re h.re - u.im h.im,  im += u.re h.im + u.im h.re
__device__ __forceinline__ void cmac16(float &ar, float &ai, uint32_t u, uint32_t h)
{
    asm("{\n\t.reg .f16 u0, u1, h0, h1, n1;\n\t"
        "mov.b32 {u0, u1}, %2;\n\tmov.b32 {h0, h1}, %3;\n\tneg.f16 n1, u1;\n\t"
        "fma.rn.f32.f16 %0, u0, h0, %0;\n\tfma.rn.f32.f16 %1, u0, h1, %1;\n\t"
        "fma.rn.f32.f16 %0, n1, h1, %0;\n\tfma.rn.f32.f16 %1, u1, h0, %1;\n\t}"
        : "+f"(ar), "+f"(ai)
        : "r"(u), "r"(h));
}
// acc += conj(u) * h:  re += u.re h.re + u.im h.im,  im += u.re h.im - u.im h.re
__device__ __forceinline__ void cjmac16(float &ar, float &ai, uint32_t u, uint32_t h)
{
    asm("{\n\t.reg .f16 u0, u1, h0, h1, n1;\n\t"
        "mov.b32 {u0, u1}, %2;\n\tmov.b32 {h0, h1}, %3;\n\tneg.f16 n1, u1;\n\t"
        "fma.rn.f32.f16 %0, u0, h0, %0;\n\tfma.rn.f32.f16 %1, u0, h1, %1;\n\t"
        "fma.rn.f32.f16 %0, u1, h1, %0;\n\tfma.rn.f32.f16 %1, n1, h0, %1;\n\t}"
        : "+f"(ar), "+f"(ai)
        : "r"(u), "r"(h));
}
// (re, im) = d * x for the real half d (the high half of dw when HI, else the low)
template <bool HI>
__device__ __forceinline__ void rmul16(float &re, float &im, uint32_t dw, uint32_t x)
{
    if (HI)
        asm("{\n\t.reg .f16 d0, d1, x0, x1;\n\t"
            "mov.b32 {d0, d1}, %2;\n\tmov.b32 {x0, x1}, %3;\n\t"
            "fma.rn.f32.f16 %0, d1, x0, 0f00000000;\n\tfma.rn.f32.f16 %1, d1, x1, 0f00000000;\n\t}"
            : "=f"(re), "=f"(im)
            : "r"(dw), "r"(x));
    else
        asm("{\n\t.reg .f16 d0, d1, x0, x1;\n\t"
            "mov.b32 {d0, d1}, %2;\n\tmov.b32 {x0, x1}, %3;\n\t"
            "fma.rn.f32.f16 %0, d0, x0, 0f00000000;\n\tfma.rn.f32.f16 %1, d0, x1, 0f00000000;\n\t}"
            : "=f"(re), "=f"(im)
            : "r"(dw), "r"(x));
}

// a + b and a - b on packed halves, rounded to nearest
__device__ __forceinline__ uint32_t h2_add(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("add.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}
__device__ __forceinline__ uint32_t h2_sub(uint32_t a, uint32_t b)
{
    uint32_t d;
    asm("sub.rn.f16x2 %0, %1, %2;" : "=r"(d) : "r"(a), "r"(b));
    return d;
}

// z + i w and z - i w on packed halves: w's halves swapped and scaled by
// (-1, 1) or (1, -1) in one FP16x2 multiply-add (the factors are exact, so the
// result is z + (-Im w, Re w), or z + (Im w, -Re w), rounded once)
__device__ __forceinline__ uint32_t h2_add_iw(uint32_t z, uint32_t w)
{
    uint32_t d;
    asm("{\n\t.reg .b16 w0, w1;\n\t.reg .b32 sw;\n\t"
        "mov.b32 {w0, w1}, %2;\n\tmov.b32 sw, {w1, w0};\n\tfma.rn.f16x2 %0, sw, %3, %1;\n\t}"
        : "=r"(d)
        : "r"(z), "r"(w), "r"(0x3C00BC00u));
    return d;
}
__device__ __forceinline__ uint32_t h2_sub_iw(uint32_t z, uint32_t w)
{
    uint32_t d;
    asm("{\n\t.reg .b16 w0, w1;\n\t.reg .b32 sw;\n\t"
        "mov.b32 {w0, w1}, %2;\n\tmov.b32 sw, {w1, w0};\n\tfma.rn.f16x2 %0, sw, %3, %1;\n\t}"
        : "=r"(d)
        : "r"(z), "r"(w), "r"(0xBC003C00u));
    return d;
}

// Spin projection (1 + SGN gamma_mu) psi on packed halves, psi[spin*3 + colour]:
//   spatial: h = psi_u - SGN i s_k psi_l;  time: h = psi_u - SGN psi_l,
// with i s_x (a, b) = (i b, i a), i s_y (a, b) = (b, -a), i s_z (a, b) = (i a, -i b).
template <int MU, int SGN>
__device__ __forceinline__ void project16(const uint32_t s[12], uint32_t h[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const uint32_t a = s[6 + c], b = s[9 + c];
        if (MU == 0) {
            h[c] = SGN > 0 ? h2_sub_iw(s[c], b) : h2_add_iw(s[c], b);
            h[3 + c] = SGN > 0 ? h2_sub_iw(s[3 + c], a) : h2_add_iw(s[3 + c], a);
        }
        if (MU == 1) {
            h[c] = SGN > 0 ? h2_sub(s[c], b) : h2_add(s[c], b);
            h[3 + c] = SGN > 0 ? h2_add(s[3 + c], a) : h2_sub(s[3 + c], a);
        }
        if (MU == 2) {
            h[c] = SGN > 0 ? h2_sub_iw(s[c], a) : h2_add_iw(s[c], a);
            h[3 + c] = SGN > 0 ? h2_add_iw(s[3 + c], b) : h2_sub_iw(s[3 + c], b);
        }
        if (MU == 3) {
            h[c] = SGN > 0 ? h2_sub(s[c], a) : h2_add(s[c], a);
            h[3 + c] = SGN > 0 ? h2_sub(s[3 + c], b) : h2_add(s[3 + c], b);
        }
    }
}

// w = U h (DAG false) or U^dagger h (DAG true) for the two colour vectors of h;
// u[row*3 + col] packed halves, w in FP32
template <bool DAG>
__device__ __forceinline__ void su3_mul16(const uint32_t u[9], const uint32_t h[6], float wr[6], float wi[6])
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            float ar = 0.f, ai = 0.f;
#pragma unroll
            for (int b = 0; b < 3; ++b) {
                if (DAG) cjmac16(ar, ai, u[b * 3 + a], h[3 * s + b]);
                else cmac16(ar, ai, u[a * 3 + b], h[3 * s + b]);
            }
            wr[3 * s + a] = ar;
            wi[3 * s + a] = ai;
        }
}

// row 2 of an SU(3) link from rows 0 and 1, row2 = conj(row0 x row1), formed
// with exact FP16 products and FP32 sums, rounded once to FP16 (the precision
// in which an uncompressed FP16 link stores it)
__device__ __forceinline__ void row2_16(uint32_t u[9])
{
    // conj(a b - c d):  re = a.re b.re - a.im b.im - c.re d.re + c.im d.im,
    //                   im = -a.re b.im - a.im b.re + c.re d.im + c.im d.re
    auto entry = [](uint32_t a, uint32_t b, uint32_t c, uint32_t d) {
        float re, im;
        asm("{\n\t.reg .f16 a0, a1, b0, b1, c0, c1, d0, d1, na0, na1, nc0;\n\t"
            "mov.b32 {a0, a1}, %2;\n\tmov.b32 {b0, b1}, %3;\n\tmov.b32 {c0, c1}, %4;\n\tmov.b32 {d0, d1}, %5;\n\t"
            "neg.f16 na0, a0;\n\tneg.f16 na1, a1;\n\tneg.f16 nc0, c0;\n\t"
            "fma.rn.f32.f16 %0, a0, b0, 0f00000000;\n\tfma.rn.f32.f16 %1, na0, b1, 0f00000000;\n\t"
            "fma.rn.f32.f16 %0, na1, b1, %0;\n\tfma.rn.f32.f16 %1, na1, b0, %1;\n\t"
            "fma.rn.f32.f16 %0, nc0, d0, %0;\n\tfma.rn.f32.f16 %1, c0, d1, %1;\n\t"
            "fma.rn.f32.f16 %0, c1, d1, %0;\n\tfma.rn.f32.f16 %1, c1, d0, %1;\n\t}"
            : "=f"(re), "=f"(im)
            : "r"(a), "r"(b), "r"(c), "r"(d));
        return pack_half2(re, im);
    };
    u[6] = entry(u[1], u[5], u[2], u[4]);
    u[7] = entry(u[2], u[3], u[0], u[5]);
    u[8] = entry(u[0], u[4], u[1], u[3]);
}

// acc += coef * (the four-spinor reconstructed from w) for the projector
// 1 + SGN gamma_mu (the lower spins are SGN i s_k w, or -SGN w in time)
template <int MU, int SGN>
__device__ __forceinline__ void reconstruct16(float ar[12], float ai[12], const float wr[6], const float wi[6],
                                              float coef)
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        const float w0r = wr[c], w0i = wi[c], w1r = wr[3 + c], w1i = wi[3 + c];
        ar[c] = fmaf(coef, w0r, ar[c]);
        ai[c] = fmaf(coef, w0i, ai[c]);
        ar[3 + c] = fmaf(coef, w1r, ar[3 + c]);
        ai[3 + c] = fmaf(coef, w1i, ai[3 + c]);
        // (o0, o1) = i s_k (w0, w1), or (w0, w1) in time; lower = s * (o0, o1)
        const float s = (MU == 3) ? (SGN > 0 ? -coef : coef) : (SGN > 0 ? coef : -coef);
        float o0r, o0i, o1r, o1i;
        if (MU == 0) { o0r = -w1i; o0i = w1r; o1r = -w0i; o1i = w0r; }
        if (MU == 1) { o0r = w1r; o0i = w1i; o1r = -w0r; o1i = -w0i; }
        if (MU == 2) { o0r = -w0i; o0i = w0r; o1r = w1i; o1i = -w1r; }
        if (MU == 3) { o0r = w0r; o0i = w0i; o1r = w1r; o1i = w1i; }
        ar[6 + c] = fmaf(s, o0r, ar[6 + c]);
        ai[6 + c] = fmaf(s, o0i, ai[6 + c]);
        ar[9 + c] = fmaf(s, o1r, ar[9 + c]);
        ai[9 + c] = fmaf(s, o1i, ai[9 + c]);
    }
}

// o += s * C_chi x for one chiral block on packed halves: b[18] its clover
// words (three words of diagonal pairs, then the 15 entries below the diagonal
// in row order), x[6] the spinor words of its two spins, s the product of the
// two scales; o in FP32
__device__ __forceinline__ void clover_block16(const uint32_t b[18], const uint32_t x[6], float s, float o_r[6],
                                               float o_i[6])
{
    float tr[6], ti[6];
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        if (a & 1) rmul16<true>(tr[a], ti[a], b[a >> 1], x[a]);
        else rmul16<false>(tr[a], ti[a], b[a >> 1], x[a]);
    }
    int k = 3;
#pragma unroll
    for (int a = 1; a < 6; ++a)
#pragma unroll
        for (int c = 0; c < a; ++c) {
            const uint32_t L = b[k++];
            cmac16(tr[a], ti[a], L, x[c]);   // L_ac x_c
            cjmac16(tr[c], ti[c], L, x[a]);  // conj(L_ac) x_a
        }
#pragma unroll
    for (int a = 0; a < 6; ++a) {
        o_r[a] = fmaf(s, tr[a], o_r[a]);
        o_i[a] = fmaf(s, ti[a], o_i[a]);
    }
}

// o += s C v for the clover term whose nine 16-byte planes start at q with a
// stride of `stride` uint4 (global memory when LDG, else shared), one chiral
// block (words 18 chi .. 18 chi + 17) at a time
template <bool LDG>
__device__ __forceinline__ void clover_planes16(const uint4 *q, size_t stride, const uint32_t v[12], float s,
                                                float ar[12], float ai[12])
{
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        uint32_t b[18];
#pragma unroll
        for (int k = 0; k < 5; ++k) {
            const uint4 w = LDG ? __ldg(q + (4 * chi + k) * stride) : q[(4 * chi + k) * stride];
            const uint32_t ws[4] = {w.x, w.y, w.z, w.w};
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                const int idx = 4 * (4 * chi + k) + e - 18 * chi;
                if (idx >= 0 && idx < 18) b[idx] = ws[e];
            }
        }
        clover_block16(b, v + 6 * chi, s, ar + 6 * chi, ai + 6 * chi);
    }
}

// ---- operands read from global memory (the packed FP16 fields)

// the stored halves of U_mu(i), u[row*3 + col]; 12-real links rebuild row 2
__device__ __forceinline__ void links16(const Gauge16x18 &U, int i, int mu, uint32_t u[9])
{
    const uint32_t *q = U.p + (((size_t)(i >> U.lvb) * 4 + mu) * 9 << U.lvb) + (i & ((1 << U.lvb) - 1));
#pragma unroll
    for (int k = 0; k < 9; ++k) u[k] = __ldg(q + ((size_t)k << U.lvb));
}
__device__ __forceinline__ void links16(const Gauge16x12 &U, int i, int mu, uint32_t u[9])
{
    const uint2 *q = U.p + (((size_t)(i >> U.lvb) * 4 + mu) * 3 << U.lvb) + (i & ((1 << U.lvb) - 1));
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint2 v = __ldg(q + ((size_t)k << U.lvb));
        u[2 * k] = v.x;
        u[2 * k + 1] = v.y;
    }
    row2_16(u);
}

// the twelve stored words of spinor site i
__device__ __forceinline__ void words16(const Spinor16 &S, int i, uint32_t w[12])
{
    const uint4 *q = S.at(i);
#pragma unroll
    for (int k = 0; k < 3; ++k) {
        const uint4 v = __ldg(q + ((size_t)k << S.lvb));
        w[4 * k] = v.x;
        w[4 * k + 1] = v.y;
        w[4 * k + 2] = v.z;
        w[4 * k + 3] = v.w;
    }
}

// o += s C(i) v at site i of the packed FP16 clover field
__device__ __forceinline__ void clover16_site(const Clover16 &C, int i, const uint32_t v[12], float s, float ar[12],
                                              float ai[12])
{
    const uint4 *q = C.p + ((size_t)(i >> C.lvb) * 9 << C.lvb) + (i & ((1 << C.lvb) - 1));
    clover_planes16<true>(q, (size_t)1 << C.lvb, v, s, ar, ai);
}

// acc += mk (the hop from x + mu along MU) with the link words u of U_mu(x),
// the neighbour's scale and the t-boundary sign in the coefficient
template <int MU, bool DAG>
__device__ __forceinline__ void hop16_fwd_u(const Geom &g, const int c[4], const Spinor16 &in, const uint32_t u[9],
                                            float mk, float ar[12], float ai[12])
{
    constexpr int SF = DAG ? +1 : -1;
    bool wr;
    uint32_t s[12], h[6];
    float wre[6], wim[6];
    const int j = neighbour(g, c, MU, +1, &wr);
    words16(in, j, s);
    float coef = mk * in.scale_of(j);
    if (MU == 3 && wr && g.tbc < 0) coef = -coef;
    project16<MU, SF>(s, h);
    su3_mul16<false>(u, h, wre, wim);
    reconstruct16<MU, SF>(ar, ai, wre, wim, coef);
}

// acc += mk (the hop from x - mu along MU), U_mu(x - mu) from global memory
template <int MU, bool DAG, class GA>
__device__ __forceinline__ void hop16_back(const Geom &g, const int c[4], const Spinor16 &in, const GA &U, float mk,
                                           float ar[12], float ai[12])
{
    constexpr int SB = DAG ? -1 : +1;
    bool wr;
    uint32_t s[12], h[6], u[9];
    float wre[6], wim[6];
    const int j = neighbour(g, c, MU, -1, &wr);
    words16(in, j, s);
    float coef = mk * in.scale_of(j);
    if (MU == 3 && wr && g.tbc < 0) coef = -coef;
    project16<MU, SB>(s, h);
    links16(U, j, MU, u);
    su3_mul16<true>(u, h, wre, wim);
    reconstruct16<MU, SB>(ar, ai, wre, wim, coef);
}

// acc += -kappa (the two hops along MU), each with its neighbour's scale and
// the t-boundary sign in the coefficient
template <int MU, bool DAG, class GA>
__device__ __forceinline__ void hop16_dir(const Geom &g, const int c[4], int i, const Spinor16 &in, const GA &U,
                                          float mk, float ar[12], float ai[12])
{
    uint32_t u[9];
    links16(U, i, MU, u);
    hop16_fwd_u<MU, DAG>(g, c, in, u, mk, ar, ai);
    hop16_back<MU, DAG>(g, c, in, U, mk, ar, ai);
}

}  // namespace mgc
