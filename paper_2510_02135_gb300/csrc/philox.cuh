// Philox-4x32-10 counter-based generator (Salmon, Moraes, Dror & Shaw,
// "Parallel random numbers: as easy as 1, 2, 3", SC'11) and the FP64
// Box-Muller map: the library's one device definition of the noise it draws
// (Lanczos W, RFD displacements, batched Brownian noise).
//
// A Philox round maps the counter (c0, c1, c2, c3) with key (k0, k1) to
//   (hi(M1 c2) ^ c1 ^ k0, lo(M1 c2), hi(M0 c0) ^ c3 ^ k1, lo(M0 c0)),
// M0 = 0xD2511F53, M1 = 0xCD9E8D57; the key is bumped by the Weyl constants
// (0x9E3779B9, 0xBB67AE85) after every round but the last; 10 rounds.
#pragma once

#include <cuda_runtime.h>

#include <cstdint>

namespace lmk {

__device__ __forceinline__ void philox4x32_10(uint32_t c[4], uint32_t k0, uint32_t k1) {
    constexpr uint32_t M0 = 0xD2511F53u, M1 = 0xCD9E8D57u, W0 = 0x9E3779B9u, W1 = 0xBB67AE85u;
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint32_t hi0 = __umulhi(M0, c[0]), lo0 = M0 * c[0];
        const uint32_t hi1 = __umulhi(M1, c[2]), lo1 = M1 * c[2];
        const uint32_t n0 = hi1 ^ c[1] ^ k0, n1 = lo1, n2 = hi0 ^ c[3] ^ k1, n3 = lo0;
        c[0] = n0; c[1] = n1; c[2] = n2; c[3] = n3;
        if (r < 9) { k0 += W0; k1 += W1; }
    }
}

// Four standard normals of counter block q of a stream: counter
// (q low, q high, stream low, stream high), key (seed low, seed high);
// normals 0, 1 from words (0, 1) and 2, 3 from words (2, 3) by Box-Muller:
// u1 = (w0 + 1) / 2^32 in (0, 1], u2 = w1 / 2^32,
// z = sqrt(-2 ln u1) (cos 2 pi u2, sin 2 pi u2).
__device__ __forceinline__ void philox_normals4(uint64_t seed, uint64_t stream, uint64_t q, double z[4]) {
    uint32_t c[4] = {(uint32_t)(q & 0xffffffffu), (uint32_t)(q >> 32), (uint32_t)(stream & 0xffffffffu),
                     (uint32_t)(stream >> 32)};
    philox4x32_10(c, (uint32_t)(seed & 0xffffffffu), (uint32_t)(seed >> 32));
#pragma unroll
    for (int p = 0; p < 2; ++p) {
        const double u1 = ((double)c[2 * p] + 1.0) * (1.0 / 4294967296.0);
        const double u2 = (double)c[2 * p + 1] * (1.0 / 4294967296.0);
        const double rad = sqrt(-2.0 * log(u1));
        double sn, cs;
        sincospi(2.0 * u2, &sn, &cs);
        z[2 * p] = rad * cs;
        z[2 * p + 1] = rad * sn;
    }
}

}  // namespace lmk
