// pm_fixed.cuh -- n keys of one length at a fixed stride (hash-table keys).
//
// Key i occupies [i * stride, i * stride + len) of the key buffer; every key
// fits in one level-1 chunk (len < m W), so its hash is the chunk value
// (b_1 + sum a_{1,i} s_i) mod p (Sec. 5, eq. 2wlinear; Sec. 6.2, Alg. 2)
// followed by the output step (Sec. 5 end, Sec. 7). One thread per key. All
// threads walk the same unit positions, so the loop is uniform (no
// predication, no second pass) and the split key words of every position are
// a uniform operand: they travel as launch parameters (constant bank). No
// offsets array is read, and outputs are stored coalesced.
#pragma once
#include "pm_lane.cuh"

namespace pm {

struct FixedParams {
    uint4 k1[M];          // split level-1 key words of unit u (64 used for n = 32, 128 for n = 64)
    uint64_t b1;          // b_1
    const uint8_t *base;  // 8-byte aligned
    uint64_t stride;      // a multiple of 8, >= len
    int64_t n;
    uint32_t len;         // < m W bytes
    void *out;            // uint32_t / uint64_t per key
};

template <int N>
__global__ void __launch_bounds__(256) k_fixed(const __grid_constant__ FixedParams P) {
    typedef typename AccT<N>::t Acc;
    const uint32_t full = P.len >> 3, rem = P.len & 7;
    const uint64_t pad = 1ull << (8 * rem);
    const int64_t stride_t = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < P.n; i += stride_t) {
        const unsigned long long *pk = reinterpret_cast<const unsigned long long *>(P.base + (uint64_t)i * P.stride);
        Acc acc;
        acc.zero();
        uint32_t u = 0;
        // four units per step: the loads of a step are issued together
        for (; u + 4 <= full; u += 4) {
            const uint64_t x0 = __ldg(pk + u), x1 = __ldg(pk + u + 1), x2 = __ldg(pk + u + 2), x3 = __ldg(pk + u + 3);
            mac_unit(acc, P.k1[u], x0);
            mac_unit(acc, P.k1[u + 1], x1);
            mac_unit(acc, P.k1[u + 2], x2);
            mac_unit(acc, P.k1[u + 3], x3);
        }
        for (; u < full; ++u) mac_unit(acc, P.k1[u], __ldg(pk + u));
        // the tail unit: the last len % 8 bytes and the 0x01 pad of Sec. 4
        const uint64_t w = rem ? __ldg(pk + full) : 0ull;
        mac_unit(acc, P.k1[full], (w & (pad - 1)) | pad);
        write_output<N>(P.out, nullptr, (uint64_t)i, acc.finish(P.b1));
    }
}

}  // namespace pm
