// Seeded Gaussian projections g_{a,l} (Sec. 3.4), host side.
//
// Philox-4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): 10 rounds of
// (hi0, lo0) = M0 * c0, (hi1, lo1) = M1 * c2,
// c <- (hi1 ^ c1 ^ k0, lo1, hi0 ^ c3 ^ k1, lo0), key bumped by the Weyl
// constants between rounds.  Box-Muller turns two uint32 draws into two
// standard normals.  Projection l of anchor length a, dimensions 4c..4c+3,
// is drawn from counter (c, l, a, 0x50414E43) under key
// (seed mod 2^32, seed div 2^32); l = B + 1 is the sieve direction.
#pragma once
#include <math.h>
#include <stdint.h>

namespace pn {

inline void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = (uint64_t)0xD2511F53u * c[0];
        const uint64_t p1 = (uint64_t)0xCD9E8D57u * c[2];
        const uint32_t n0 = (uint32_t)(p1 >> 32) ^ c[1] ^ k0;
        const uint32_t n1 = (uint32_t)p1;
        const uint32_t n2 = (uint32_t)(p0 >> 32) ^ c[3] ^ k1;
        const uint32_t n3 = (uint32_t)p0;
        c[0] = n0;
        c[1] = n1;
        c[2] = n2;
        c[3] = n3;
        if (r < 9) {
            k0 += 0x9E3779B9u;
            k1 += 0xBB67AE85u;
        }
    }
}

// rows [B+1][32] floats; dims >= 2(K-1) are zero.
inline void projections(int a, uint64_t seed, int B, int K, float *out) {
    const int dims = 2 * (K - 1);
    const int groups = (dims + 3) / 4;
    const double two_pi = 6.283185307179586476925286766559;
    for (int l = 1; l <= B + 1; ++l) {
        float *row = out + (l - 1) * 32;
        for (int t = 0; t < 32; ++t) row[t] = 0.0f;
        for (int c = 0; c < groups; ++c) {
            uint32_t ctr[4] = {(uint32_t)c, (uint32_t)l, (uint32_t)a, 0x50414E43u};
            philox4x32_10(ctr, (uint32_t)(seed & 0xFFFFFFFFu), (uint32_t)(seed >> 32));
            for (int h = 0; h < 2; ++h) {
                const double u = ((double)ctr[2 * h] + 1.0) * (1.0 / 4294967296.0);
                const double w = (double)ctr[2 * h + 1] * (1.0 / 4294967296.0);
                const double r = sqrt(-2.0 * log(u));
                const int d0 = 4 * c + 2 * h;
                if (d0 < dims) row[d0] = (float)(r * cos(two_pi * w));
                if (d0 + 1 < dims) row[d0 + 1] = (float)(r * sin(two_pi * w));
            }
        }
    }
}

}  // namespace pn
