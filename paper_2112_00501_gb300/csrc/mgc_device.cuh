// Device-side building blocks: lattice geometry of the packed layout, complex
// arithmetic, per-precision field accessors, and the spin projection /
// reconstruction of the Wilson hopping term in the chiral gamma basis.
//
// Packed site order: i = blk * Vb + l, with blk the SAP domain (block) index
// (x fastest) and l = parity * Vb/2 + h inside the block, where parity is the
// site parity and h = (lx >> 1) + (Bx/2) * (ly + By * (lz + Bz * lt)).  Block
// extents are powers of two >= 2, so l and the local coordinates convert with
// shifts and masks.
#pragma once

#include <cfloat>
#include <cuda_fp16.h>
#include <cuda_runtime.h>
#include <stdint.h>

namespace mgc {

struct Geom {
    int L[4];   // lattice extents x, y, z, t
    int NB[4];  // blocks per direction
    int lb[4];  // log2 of the block extents
    int lvb;    // log2 of sites per block
    int nblocks;
    int V;      // sites
    int tbc;    // +1 periodic, -1 antiperiodic in t
};

// ------------------------------------------------------------------ complex
template <typename T>
struct Cx {
    T r, i;
};

template <typename T>
__device__ __forceinline__ Cx<T> mk(T r, T i) { return Cx<T>{r, i}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator+(Cx<T> a, Cx<T> b) { return {a.r + b.r, a.i + b.i}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator-(Cx<T> a, Cx<T> b) { return {a.r - b.r, a.i - b.i}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator-(Cx<T> a) { return {-a.r, -a.i}; }
template <typename T>
__device__ __forceinline__ Cx<T> operator*(Cx<T> a, Cx<T> b)
{
    return {a.r * b.r - a.i * b.i, a.r * b.i + a.i * b.r};
}
template <typename T>
__device__ __forceinline__ Cx<T> operator*(T s, Cx<T> a) { return {s * a.r, s * a.i}; }
template <typename T>
__device__ __forceinline__ Cx<T> conj(Cx<T> a) { return {a.r, -a.i}; }
// a * b + c
template <typename T>
__device__ __forceinline__ Cx<T> cfma(Cx<T> a, Cx<T> b, Cx<T> c)
{
    return {fma(a.r, b.r, fma(-a.i, b.i, c.r)), fma(a.r, b.i, fma(a.i, b.r, c.i))};
}
// conj(a) * b + c
template <typename T>
__device__ __forceinline__ Cx<T> cjfma(Cx<T> a, Cx<T> b, Cx<T> c)
{
    return {fma(a.r, b.r, fma(a.i, b.i, c.r)), fma(a.r, b.i, fma(-a.i, b.r, c.i))};
}
template <typename T>
__device__ __forceinline__ Cx<T> times_i(Cx<T> a) { return {-a.i, a.r}; }
template <typename T>
__device__ __forceinline__ T norm2(Cx<T> a) { return a.r * a.r + a.i * a.i; }

// ------------------------------------------------------------------ geometry
__device__ __forceinline__ void local_coords(const Geom &g, int l, int lc[4])
{
    const int hb = g.lvb - 1;
    const int par = l >> hb;
    const int h = l & ((1 << hb) - 1);
    const int sx = g.lb[0] - 1;
    int rest = h >> sx;
    lc[1] = rest & ((1 << g.lb[1]) - 1);
    rest >>= g.lb[1];
    lc[2] = rest & ((1 << g.lb[2]) - 1);
    lc[3] = rest >> g.lb[2];
    const int xlo = (par + lc[1] + lc[2] + lc[3]) & 1;
    lc[0] = ((h & ((1 << sx) - 1)) << 1) | xlo;
}

__device__ __forceinline__ int local_index(const Geom &g, const int lc[4])
{
    const int par = (lc[0] + lc[1] + lc[2] + lc[3]) & 1;
    const int h = (lc[0] >> 1) + ((lc[1] + ((lc[2] + (lc[3] << g.lb[2])) << g.lb[1])) << (g.lb[0] - 1));
    return (par << (g.lvb - 1)) | h;
}

__device__ __forceinline__ void block_coords(const Geom &g, int blk, int bc[4])
{
    bc[0] = blk % g.NB[0];
    blk /= g.NB[0];
    bc[1] = blk % g.NB[1];
    blk /= g.NB[1];
    bc[2] = blk % g.NB[2];
    bc[3] = blk / g.NB[2];
}

__device__ __forceinline__ int block_index(const Geom &g, const int bc[4])
{
    return bc[0] + g.NB[0] * (bc[1] + g.NB[1] * (bc[2] + g.NB[2] * bc[3]));
}

// global coordinates of packed site i
__device__ __forceinline__ void site_coords(const Geom &g, int i, int c[4])
{
    int lc[4], bc[4];
    local_coords(g, i & ((1 << g.lvb) - 1), lc);
    block_coords(g, i >> g.lvb, bc);
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) c[mu] = (bc[mu] << g.lb[mu]) + lc[mu];
}

// packed index of the site with global coordinates c (each in range)
__device__ __forceinline__ int site_index(const Geom &g, const int c[4])
{
    int lc[4], bc[4];
#pragma unroll
    for (int mu = 0; mu < 4; ++mu) {
        bc[mu] = c[mu] >> g.lb[mu];
        lc[mu] = c[mu] & ((1 << g.lb[mu]) - 1);
    }
    return (block_index(g, bc) << g.lvb) | local_index(g, lc);
}

// canonical (lexicographic) index of global coordinates c
__device__ __forceinline__ long long canon_index(const Geom &g, const int c[4])
{
    return c[0] + (long long)g.L[0] * (c[1] + (long long)g.L[1] * (c[2] + (long long)g.L[2] * c[3]));
}

// neighbour of c in direction mu (dir = +1/-1) with periodic wrap;
// returns its packed index and sets *wrapped when the hop crosses the boundary
__device__ __forceinline__ int neighbour(const Geom &g, const int c[4], int mu, int dir, bool *wrapped)
{
    int n[4] = {c[0], c[1], c[2], c[3]};
    int v = n[mu] + dir;
    *wrapped = false;
    if (v < 0) { v += g.L[mu]; *wrapped = true; }
    if (v >= g.L[mu]) { v -= g.L[mu]; *wrapped = true; }
    n[mu] = v;
    return site_index(g, n);
}

// ------------------------------------------------------------------ precisions
template <int PREC> struct RealOf { using T = float; };
template <> struct RealOf<64> { using T = double; };

// Spinor accessors: 12 complex components, index spin*3 + colour.
struct Spinor64 {
    double2 *p;
    int lvb;
    using Real = double;
    __device__ __forceinline__ const double2 *at(int i) const
    {
        return p + ((size_t)(i >> lvb) * 12 << lvb) + (i & ((1 << lvb) - 1));
    }
    __device__ __forceinline__ void load(int i, Cx<double> s[12]) const
    {
        const double2 *q = at(i);
#pragma unroll
        for (int k = 0; k < 12; ++k) {
            double2 v = __ldg(q + ((size_t)k << lvb));
            s[k] = {v.x, v.y};
        }
    }
    __device__ __forceinline__ void store(int i, const Cx<double> s[12]) const
    {
        double2 *q = const_cast<double2 *>(at(i));
#pragma unroll
        for (int k = 0; k < 12; ++k) q[(size_t)k << lvb] = make_double2(s[k].r, s[k].i);
    }
};

struct Spinor32 {
    float4 *p;
    int lvb;
    using Real = float;
    __device__ __forceinline__ const float4 *at(int i) const
    {
        return p + ((size_t)(i >> lvb) * 6 << lvb) + (i & ((1 << lvb) - 1));
    }
    __device__ __forceinline__ void load(int i, Cx<float> s[12]) const
    {
        const float4 *q = at(i);
#pragma unroll
        for (int k = 0; k < 6; ++k) {
            float4 v = __ldg(q + ((size_t)k << lvb));
            s[2 * k] = {v.x, v.y};
            s[2 * k + 1] = {v.z, v.w};
        }
    }
    __device__ __forceinline__ void store(int i, const Cx<float> s[12]) const
    {
        float4 *q = const_cast<float4 *>(at(i));
#pragma unroll
        for (int k = 0; k < 6; ++k)
            q[(size_t)k << lvb] = make_float4(s[2 * k].r, s[2 * k].i, s[2 * k + 1].r, s[2 * k + 1].i);
    }
};

__device__ __forceinline__ uint32_t pack_half2(float a, float b)
{
    __half2 h = __floats2half2_rn(a, b);
    return *reinterpret_cast<uint32_t *>(&h);
}
__device__ __forceinline__ float2 unpack_half2(uint32_t u)
{
    __half2 h = *reinterpret_cast<__half2 *>(&u);
    return __half22float2(h);
}

// FP16 storage with one FP32 scale per site: value = half * scale, where the
// scale is the site's largest |real component|.
struct Spinor16 {
    uint4 *p;
    float *sc;
    int lvb;
    using Real = float;
    __device__ __forceinline__ const uint4 *at(int i) const
    {
        return p + ((size_t)(i >> lvb) * 3 << lvb) + (i & ((1 << lvb) - 1));
    }
    // the stored halves without the scale, and the scale
    __device__ __forceinline__ void load_raw(int i, Cx<float> s[12]) const
    {
        const uint4 *q = at(i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(q + ((size_t)k << lvb));
            float2 a = unpack_half2(v.x), b = unpack_half2(v.y), c = unpack_half2(v.z), d = unpack_half2(v.w);
            s[4 * k + 0] = {a.x, a.y};
            s[4 * k + 1] = {b.x, b.y};
            s[4 * k + 2] = {c.x, c.y};
            s[4 * k + 3] = {d.x, d.y};
        }
    }
    __device__ __forceinline__ float scale_of(int i) const { return __ldg(sc + i); }
    __device__ __forceinline__ void load(int i, Cx<float> s[12]) const
    {
        const uint4 *q = at(i);
        const float scale = __ldg(sc + i);
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v = __ldg(q + ((size_t)k << lvb));
            float2 a = unpack_half2(v.x), b = unpack_half2(v.y), c = unpack_half2(v.z), d = unpack_half2(v.w);
            s[4 * k + 0] = {a.x * scale, a.y * scale};
            s[4 * k + 1] = {b.x * scale, b.y * scale};
            s[4 * k + 2] = {c.x * scale, c.y * scale};
            s[4 * k + 3] = {d.x * scale, d.y * scale};
        }
    }
    __device__ __forceinline__ void store(int i, const Cx<float> s[12]) const
    {
        float m = 0.f;
#pragma unroll
        for (int k = 0; k < 12; ++k) m = fmaxf(m, fmaxf(fabsf(s[k].r), fabsf(s[k].i)));
        const float inv = (m >= FLT_MIN) ? 1.0f / m : 0.f;  // a site below FP32's normal range is stored as zero
        uint4 *q = const_cast<uint4 *>(at(i));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint4 v;
            v.x = pack_half2(s[4 * k + 0].r * inv, s[4 * k + 0].i * inv);
            v.y = pack_half2(s[4 * k + 1].r * inv, s[4 * k + 1].i * inv);
            v.z = pack_half2(s[4 * k + 2].r * inv, s[4 * k + 2].i * inv);
            v.w = pack_half2(s[4 * k + 3].r * inv, s[4 * k + 3].i * inv);
            q[(size_t)k << lvb] = v;
        }
        sc[i] = m;
    }
};

// the rhs-th field of a batch of packed spinors (FP16 scales follow all data)
__host__ __device__ __forceinline__ Spinor64 shift_rhs(Spinor64 a, int r, int V)
{
    a.p += (size_t)r * V * 12;
    return a;
}
__host__ __device__ __forceinline__ Spinor32 shift_rhs(Spinor32 a, int r, int V)
{
    a.p += (size_t)r * V * 6;
    return a;
}
__host__ __device__ __forceinline__ Spinor16 shift_rhs(Spinor16 a, int r, int V)
{
    a.p += (size_t)r * V * 3;
    a.sc += (size_t)r * V;
    return a;
}

template <int PREC> struct SpinorOf;
template <> struct SpinorOf<64> { using type = Spinor64; };
template <> struct SpinorOf<32> { using type = Spinor32; };
template <> struct SpinorOf<16> { using type = Spinor16; };

// Gauge accessors: u[row*3 + col] of U_mu(i).  Layout per block:
// [mu][plane][site].  12-real forms keep rows 0 and 1; row 2 = conj(r0 x r1).
template <typename T>
__device__ __forceinline__ void reconstruct_row2(Cx<T> u[9])
{
    u[6] = conj(u[1] * u[5] - u[2] * u[4]);
    u[7] = conj(u[2] * u[3] - u[0] * u[5]);
    u[8] = conj(u[0] * u[4] - u[1] * u[3]);
}

struct Gauge64 {
    double2 *p;
    int lvb;
    using Real = double;
    __device__ __forceinline__ void load(int i, int mu, Cx<double> u[9]) const
    {
        const double2 *q = p + (((size_t)(i >> lvb) * 4 + mu) * 9 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            double2 v = __ldg(q + ((size_t)k << lvb));
            u[k] = {v.x, v.y};
        }
    }
};

struct Gauge32x18 {
    float2 *p;
    int lvb;
    using Real = float;
    __device__ __forceinline__ void load(int i, int mu, Cx<float> u[9]) const
    {
        const float2 *q = p + (((size_t)(i >> lvb) * 4 + mu) * 9 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 v = __ldg(q + ((size_t)k << lvb));
            u[k] = {v.x, v.y};
        }
    }
};

struct Gauge32x12 {
    float4 *p;
    int lvb;
    using Real = float;
    __device__ __forceinline__ void load(int i, int mu, Cx<float> u[9]) const
    {
        const float4 *q = p + (((size_t)(i >> lvb) * 4 + mu) * 3 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            float4 v = __ldg(q + ((size_t)k << lvb));
            u[2 * k] = {v.x, v.y};
            u[2 * k + 1] = {v.z, v.w};
        }
        reconstruct_row2(u);
    }
};

struct Gauge16x18 {
    uint32_t *p;
    int lvb;
    using Real = float;
    __device__ __forceinline__ void load(int i, int mu, Cx<float> u[9]) const
    {
        const uint32_t *q = p + (((size_t)(i >> lvb) * 4 + mu) * 9 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            float2 v = unpack_half2(__ldg(q + ((size_t)k << lvb)));
            u[k] = {v.x, v.y};
        }
    }
};

struct Gauge16x12 {
    uint2 *p;
    int lvb;
    using Real = float;
    __device__ __forceinline__ void load(int i, int mu, Cx<float> u[9]) const
    {
        const uint2 *q = p + (((size_t)(i >> lvb) * 4 + mu) * 3 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 3; ++k) {
            uint2 v = __ldg(q + ((size_t)k << lvb));
            float2 a = unpack_half2(v.x), b = unpack_half2(v.y);
            u[2 * k] = {a.x, a.y};
            u[2 * k + 1] = {b.x, b.y};
        }
        reconstruct_row2(u);
    }
};

// Clover accessors: two Hermitian 6x6 chiral blocks, 36 reals each, packed as
// 6 real diagonal entries then the 15 entries below the diagonal in row order
// (1,0) (2,0) (2,1) (3,0) ... (5,4) as (re, im).  Block 0 acts on spins 0, 1
// and block 1 on spins 2, 3.
struct Clover64 {
    double2 *p;
    int lvb;
    using Real = double;
    __device__ __forceinline__ void load(int i, double c[72]) const
    {
        const double2 *q = p + ((size_t)(i >> lvb) * 36 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 36; ++k) {
            double2 v = __ldg(q + ((size_t)k << lvb));
            c[2 * k] = v.x;
            c[2 * k + 1] = v.y;
        }
    }
};

struct Clover32 {
    float4 *p;
    int lvb;
    using Real = float;
    __device__ __forceinline__ void load(int i, float c[72]) const
    {
        const float4 *q = p + ((size_t)(i >> lvb) * 18 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 18; ++k) {
            float4 v = __ldg(q + ((size_t)k << lvb));
            c[4 * k] = v.x;
            c[4 * k + 1] = v.y;
            c[4 * k + 2] = v.z;
            c[4 * k + 3] = v.w;
        }
    }
};

struct Clover16 {
    uint4 *p;
    float *sc;
    int lvb;
    using Real = float;
    // the stored halves without the scale, and the scale
    __device__ __forceinline__ float load_raw(int i, float c[72]) const
    {
        const uint4 *q = p + ((size_t)(i >> lvb) * 9 << lvb) + (i & ((1 << lvb) - 1));
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            uint4 v = __ldg(q + ((size_t)k << lvb));
            float2 a = unpack_half2(v.x), b = unpack_half2(v.y), cc = unpack_half2(v.z), d = unpack_half2(v.w);
            c[8 * k + 0] = a.x;
            c[8 * k + 1] = a.y;
            c[8 * k + 2] = b.x;
            c[8 * k + 3] = b.y;
            c[8 * k + 4] = cc.x;
            c[8 * k + 5] = cc.y;
            c[8 * k + 6] = d.x;
            c[8 * k + 7] = d.y;
        }
        return __ldg(sc + i);
    }
    __device__ __forceinline__ void load(int i, float c[72]) const
    {
        const uint4 *q = p + ((size_t)(i >> lvb) * 9 << lvb) + (i & ((1 << lvb) - 1));
        const float s = __ldg(sc + i);
#pragma unroll
        for (int k = 0; k < 9; ++k) {
            uint4 v = __ldg(q + ((size_t)k << lvb));
            float2 a = unpack_half2(v.x), b = unpack_half2(v.y), cc = unpack_half2(v.z), d = unpack_half2(v.w);
            c[8 * k + 0] = a.x * s;
            c[8 * k + 1] = a.y * s;
            c[8 * k + 2] = b.x * s;
            c[8 * k + 3] = b.y * s;
            c[8 * k + 4] = cc.x * s;
            c[8 * k + 5] = cc.y * s;
            c[8 * k + 6] = d.x * s;
            c[8 * k + 7] = d.y * s;
        }
    }
};

// out = C in for the packed clover c[72]
template <typename T>
__device__ __forceinline__ void clover_mul(const T c[72], const Cx<T> in[12], Cx<T> out[12])
{
#pragma unroll
    for (int chi = 0; chi < 2; ++chi) {
        const T *d = c + 36 * chi;
        const Cx<T> *v = in + 6 * chi;
        Cx<T> *o = out + 6 * chi;
#pragma unroll
        for (int a = 0; a < 6; ++a) o[a] = d[a] * v[a];
        int k = 6;
#pragma unroll
        for (int a = 1; a < 6; ++a)
#pragma unroll
            for (int b = 0; b < a; ++b) {
                const Cx<T> L = {d[k], d[k + 1]};
                k += 2;
                o[a] = cfma(L, v[b], o[a]);
                o[b] = cjfma(L, v[a], o[b]);
            }
    }
}

// ------------------------------------------------------------------ hopping
// Spin projection in the chiral basis (gamma_k = [[0, -i s_k], [i s_k, 0]],
// gamma_t = [[0, -1], [-1, 0]]).  For P = 1 + SGN * gamma_mu:
//   spatial: h = psi_u - SGN i s_k psi_l; P psi = (h, SGN i s_k h)
//   time:    h = psi_u - SGN psi_l;       P psi = (h, -SGN h)
// where psi_u are spins 0, 1 and psi_l spins 2, 3.  With (a, b) a two-spin
// pair: i s_x (a, b) = (i b, i a), i s_y (a, b) = (b, -a), i s_z (a, b) = (i a, -i b).
template <int MU, typename T>
__device__ __forceinline__ void isigma(Cx<T> a, Cx<T> b, Cx<T> &o0, Cx<T> &o1)
{
    if (MU == 0) { o0 = times_i(b); o1 = times_i(a); }
    if (MU == 1) { o0 = b; o1 = -a; }
    if (MU == 2) { o0 = times_i(a); o1 = -times_i(b); }
    if (MU == 3) { o0 = a; o1 = b; }
}

template <int MU, int SGN, typename T>
__device__ __forceinline__ void project(const Cx<T> s[12], Cx<T> h[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        Cx<T> o0, o1;
        isigma<MU>(s[6 + c], s[9 + c], o0, o1);
        if (SGN > 0) { h[c] = s[c] - o0; h[3 + c] = s[3 + c] - o1; }
        else { h[c] = s[c] + o0; h[3 + c] = s[3 + c] + o1; }
    }
}

template <int MU, int SGN, typename T>
__device__ __forceinline__ void reconstruct_add(Cx<T> acc[12], const Cx<T> w[6])
{
#pragma unroll
    for (int c = 0; c < 3; ++c) {
        acc[c] = acc[c] + w[c];
        acc[3 + c] = acc[3 + c] + w[3 + c];
        if (MU == 3) {
            if (SGN > 0) { acc[6 + c] = acc[6 + c] - w[c]; acc[9 + c] = acc[9 + c] - w[3 + c]; }
            else { acc[6 + c] = acc[6 + c] + w[c]; acc[9 + c] = acc[9 + c] + w[3 + c]; }
        } else {
            Cx<T> o0, o1;
            isigma<MU>(w[c], w[3 + c], o0, o1);
            if (SGN > 0) { acc[6 + c] = acc[6 + c] + o0; acc[9 + c] = acc[9 + c] + o1; }
            else { acc[6 + c] = acc[6 + c] - o0; acc[9 + c] = acc[9 + c] - o1; }
        }
    }
}

// w = U h (two colour vectors) and w = U^dagger h
template <typename T>
__device__ __forceinline__ void su3_mul(const Cx<T> u[9], const Cx<T> h[6], Cx<T> w[6])
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Cx<T> acc = u[a * 3] * h[3 * s];
            acc = cfma(u[a * 3 + 1], h[3 * s + 1], acc);
            acc = cfma(u[a * 3 + 2], h[3 * s + 2], acc);
            w[3 * s + a] = acc;
        }
}

template <typename T>
__device__ __forceinline__ void su3_dag_mul(const Cx<T> u[9], const Cx<T> h[6], Cx<T> w[6])
{
#pragma unroll
    for (int s = 0; s < 2; ++s)
#pragma unroll
        for (int a = 0; a < 3; ++a) {
            Cx<T> acc = conj(u[a]) * h[3 * s];
            acc = cjfma(u[3 + a], h[3 * s + 1], acc);
            acc = cjfma(u[6 + a], h[3 * s + 2], acc);
            w[3 * s + a] = acc;
        }
}

template <typename T>
__device__ __forceinline__ void negate6(Cx<T> h[6])
{
#pragma unroll
    for (int k = 0; k < 6; ++k) h[k] = -h[k];
}

}  // namespace mgc
