// sigma_{mu nu} = (i/2)[gamma_mu, gamma_nu] in the chiral basis is block
// diagonal, diag(s+_{mu nu}, s-_{mu nu}); this table holds the 2x2 blocks.
#pragma once

namespace mgc {

// sigma_{mu nu} chiral 2x2 blocks, [chi][plane][s][t] as (re, im); planes in
// the order (x,y) (x,z) (x,t) (y,z) (y,t) (z,t).  Upper block: -s3, s2, -s1,
// -s1, -s2, -s3; lower block: -s3, s2, s1, -s1, s2, s3.
// (a constexpr device table: kernels that unroll over it see its entries as
// constants, so the zero entries cost nothing and the +-1, +-i ones no multiply)
static __device__ constexpr double c_sigma[2][6][2][2][2] = {
    {
        {{{-1, 0}, {0, 0}}, {{0, 0}, {1, 0}}},   // -s3
        {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},   // s2
        {{{0, 0}, {-1, 0}}, {{-1, 0}, {0, 0}}},  // -s1
        {{{0, 0}, {-1, 0}}, {{-1, 0}, {0, 0}}},  // -s1
        {{{0, 0}, {0, 1}}, {{0, -1}, {0, 0}}},   // -s2
        {{{-1, 0}, {0, 0}}, {{0, 0}, {1, 0}}},   // -s3
    },
    {
        {{{-1, 0}, {0, 0}}, {{0, 0}, {1, 0}}},   // -s3
        {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},   // s2
        {{{0, 0}, {1, 0}}, {{1, 0}, {0, 0}}},    // s1
        {{{0, 0}, {-1, 0}}, {{-1, 0}, {0, 0}}},  // -s1
        {{{0, 0}, {0, -1}}, {{0, 1}, {0, 0}}},   // s2
        {{{1, 0}, {0, 0}}, {{0, 0}, {-1, 0}}},   // s3
    },
};

}  // namespace mgc
