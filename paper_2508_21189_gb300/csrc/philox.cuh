// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11) for the device side of librsk, and the
// stream layout every random draw of the library uses:
//     word(seed, stream, entity, t) = Philox4x32-10(key = (seed_lo, seed_hi),
//                                                   ctr = (entity_lo, entity_hi, stream, t >> 2))[t & 3]
#pragma once
#include <stdint.h>

namespace rskd {

struct Block4 {
    uint32_t v[4];
};

// Ten rounds of the Philox-4x32 bijection.  Each round multiplies words 0 and 2 by the
// published constants, mixes the high halves with the other words and the round key, and the
// key is advanced by the published Weyl increments.
__host__ __device__ __forceinline__ Block4 philox4x32_10(uint32_t c0, uint32_t c1, uint32_t c2, uint32_t c3,
                                                         uint32_t k0, uint32_t k1) {
#pragma unroll
    for (int r = 0; r < 10; ++r) {
        const uint64_t p0 = uint64_t(0xD2511F53u) * c0;
        const uint64_t p1 = uint64_t(0xCD9E8D57u) * c2;
        const uint32_t n0 = uint32_t(p1 >> 32) ^ c1 ^ k0;
        const uint32_t n2 = uint32_t(p0 >> 32) ^ c3 ^ k1;
        c1 = uint32_t(p1);
        c3 = uint32_t(p0);
        c0 = n0;
        c2 = n2;
        k0 += 0x9E3779B9u;
        k1 += 0xBB67AE85u;
    }
    Block4 b;
    b.v[0] = c0;
    b.v[1] = c1;
    b.v[2] = c2;
    b.v[3] = c3;
    return b;
}

// Four consecutive words t = 4*blk .. 4*blk+3 of (seed, stream, entity).
__host__ __device__ __forceinline__ Block4 philox_block(uint64_t seed, uint32_t stream, uint64_t entity,
                                                        uint32_t blk) {
    return philox4x32_10(uint32_t(entity), uint32_t(entity >> 32), stream, blk, uint32_t(seed),
                         uint32_t(seed >> 32));
}

}  // namespace rskd
