// pm_fixed.cuh -- n keys of one length at a fixed stride (hash-table keys).
//
// Key i occupies [i * stride, i * stride + len) of the key buffer; every key
// fits in one level-1 chunk (len < m W), so its hash is the chunk value
// (b_1 + sum a_{1,i} s_i) mod p (Sec. 5, eq. 2wlinear; Sec. 6.2, Alg. 2)
// followed by the output step (Sec. 5 end, Sec. 7). Three kernels by length:
//   k_fixed_one (at most 8 bytes): one unit, a full product per word with
//     explicit carries, the pad's constant folded into b_1;
//   k_fixed_few (2..9 units, up to 72 bytes): every unit on carry chains,
//     the key words of the unit positions as launch parameters;
//   k_fixed (longer keys): one thread per key, four units per step, split
//     key words.
// The first two take two keys per thread (i, i + T for T threads, so that
// every load instruction of a warp reads consecutive keys), their loads
// issued before the multiply-adds: one short key per thread leaves too few
// bytes in flight to cover the memory latency. All threads walk the same unit
// positions, so the loops are uniform (no predication, no second pass), and
// the key words of every position are uniform operands (constant bank). No
// offsets array is read, and outputs are stored coalesced.
#pragma once
#include "pm_lane.cuh"

namespace pm {

struct FixedParams {
    uint4 k1[M];          // split level-1 key words of unit u (64 used for n = 32, 128 for n = 64)
    uint64_t b1;          // b_1
    // keys of at most 8 bytes (k_fixed_one): the key words of unit 0 (n = 32:
    // a_1, a_2; n = 64: a_1) and c = b_1 + the key word that weighs the pad
    // word when len == 8 (the unit after the key is the word 1), c_lo + 2^64 c_hi
    uint64_t a0, a1, c_lo, c_hi;
    // keys of 2..FIXED_FEW_MAX units (k_fixed_few): the key words of units
    // 0..FIXED_FEW_MAX-1 (n = 32: a_{2u+1} | a_{2u+2} << 32; n = 64: a_{u+1})
    // and, when len % 8 == 0, the key word that weighs the pad word 1 (else 0)
    uint64_t kw[9], pad_kw;
    const uint8_t *base;  // 8-byte aligned
    uint64_t stride;      // a multiple of 8, >= len
    int64_t n;
    uint32_t len;         // < m W bytes
    void *out;            // uint32_t / uint64_t per key
};

// acc += k * 1 for a unit that is the pad alone (first word 1, the rest 0):
// the same sums as mac_unit(acc, k, 1) without the multiplies.
__device__ __forceinline__ void add_pad_unit(Acc32 &acc, const uint4 &k) {
    acc.L += k.x;
    acc.H += k.y;
}
__device__ __forceinline__ void add_pad_unit(Acc64 &acc, const uint4 &k) {
    acc.a00 += k.x;
    acc.a10 += k.y;
    acc.a20 += k.z;
}

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
        if (rem)
            mac_unit(acc, P.k1[full], (__ldg(pk + full) & (pad - 1)) | pad);
        else
            add_pad_unit(acc, P.k1[full]);  // the unit is the word 1: its key word alone
        write_output<N>(P.out, nullptr, (uint64_t)i, acc.finish(P.b1));
    }
}

// (c + sum of the key words times the words of the one unit x) mod p for a
// key of at most 8 bytes: a single 32 x 32 or 64 x 64 multiply per word,
// carries added explicitly, then Sec. 6.2 and Alg. 2.
__device__ __forceinline__ Val one_unit_value(const FixedParams &P, uint64_t x, Fam<32>) {
    // the key words are below 2^32: one 32 x 32 -> 64 multiply each
    const uint64_t p0 = (uint64_t)(uint32_t)P.a0 * (uint32_t)x, p1 = (uint64_t)(uint32_t)P.a1 * (uint32_t)(x >> 32);
    const uint64_t t = p0 + p1;
    const uint64_t u = t + P.c_lo;  // c < 2^33
    const uint32_t w2 = (uint32_t)(t < p0) + (uint32_t)(u < t);
    return reduce32_limbs((uint32_t)u, (uint32_t)(u >> 32), w2);
}
__device__ __forceinline__ Val one_unit_value(const FixedParams &P, uint64_t x, Fam<64>) {
    const uint64_t lo = P.a0 * x, hi = __umul64hi(P.a0, x);
    const uint64_t w0 = lo + P.c_lo;
    const uint64_t h1 = hi + P.c_hi;  // c < 2^65
    const uint64_t w1 = h1 + (uint64_t)(w0 < lo);
    const uint64_t w2 = (uint64_t)(h1 < hi) + (uint64_t)(w1 < h1);
    return reduce64(w0, w1, w2);
}

// Keys of at most 8 bytes: the unit holds the key's bytes and, when len < 8,
// the 0x01 pad of Sec. 4; when len == 8 the pad is the next unit, the word 1,
// whose product is the constant folded into c. Two keys per thread (i,
// i + T), their loads issued together (one, four and eight keys, and two
// adjacent keys in one 16-byte load, measured slower); a 0-byte key reads
// nothing.
template <int N>
__global__ void __launch_bounds__(256) k_fixed_one(const __grid_constant__ FixedParams P) {
    constexpr int K = 2;
    const uint32_t len = P.len;
    const uint64_t padbit = len < 8 ? 1ull << (8 * len) : 0ull;
    const uint64_t mask = len < 8 ? padbit - 1 : ~0ull;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < P.n; i0 += K * T) {
        uint64_t x[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t i = i0 + j * T;
            x[j] = len && i < P.n
                       ? __ldg(reinterpret_cast<const unsigned long long *>(P.base + (uint64_t)i * P.stride))
                       : 0ull;
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t i = i0 + j * T;
            if (i < P.n) write_output<N>(P.out, nullptr, (uint64_t)i, one_unit_value(P, (x[j] & mask) | padbit, Fam<N>()));
        }
    }
}

constexpr int FIXED_FEW_MAX = 9;  // units of the longest keys of k_fixed_few (72 bytes)

// Keys of 2..U units (9..8U bytes): every unit a full product per word on
// carry chains (the key words of a unit position are launch parameters), the
// tail unit masked with the 0x01 pad of Sec. 4, or, when len % 8 == 0, the pad
// word's key word added once; then Sec. 6.2, Alg. 2 and the output step. Two
// keys per thread (i, i + T), all their loads issued first; with V16 (a
// 16-byte aligned buffer and a stride of a multiple of 64 bytes) two units
// per 16-byte load.
template <int N, int U, bool V16>
__global__ void __launch_bounds__(256) k_fixed_few(const __grid_constant__ FixedParams P) {
    typedef typename AccCT<N>::t AccC;
    constexpr int K = 2;
    const uint32_t full = P.len >> 3, rem = P.len & 7;
    const uint32_t nu = full + (rem ? 1u : 0u);  // units read
    const uint64_t padbit = rem ? 1ull << (8 * rem) : 0ull;
    const uint64_t mask = rem ? padbit - 1 : ~0ull;
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < P.n; i0 += K * T) {
        uint64_t x[K][U];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t i = i0 + j * T;
            const unsigned long long *pk = reinterpret_cast<const unsigned long long *>(P.base + (uint64_t)i * P.stride);
            if constexpr (V16) {  // 16-byte aligned keys: two units per load
                const ulonglong2 *pv = reinterpret_cast<const ulonglong2 *>(pk);
#pragma unroll
                for (int u = 0; u < U; u += 2) {
                    if ((uint32_t)u + 1 < nu && i < P.n) {
                        const ulonglong2 v = __ldg(pv + u / 2);
                        x[j][u] = v.x;
                        if (u + 1 < U) x[j][u + 1] = v.y;
                    } else {
                        x[j][u] = (uint32_t)u < nu && i < P.n ? __ldg(pk + u) : 0ull;
                        if (u + 1 < U) x[j][u + 1] = 0ull;
                    }
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) x[j][u] = (uint32_t)u < nu && i < P.n ? __ldg(pk + u) : 0ull;
            }
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t i = i0 + j * T;
            AccC acc;
            acc.zero();
#pragma unroll
            for (int u = 0; u < U; ++u) {
                uint64_t xu = x[j][u];
                if ((uint32_t)u == full && rem) xu = (xu & mask) | padbit;  // the tail unit
                if ((uint32_t)u < nu) {
                    if constexpr (N == 32)
                        add_unit_c(acc, make_uint2((uint32_t)P.kw[u], (uint32_t)(P.kw[u] >> 32)), xu);
                    else
                        add_unit_c(acc, P.kw[u], xu);
                }
            }
            if (!rem) {  // the pad word 1 after the whole units
                if constexpr (N == 32)
                    acc.add((uint32_t)P.pad_kw, 1u);
                else
                    acc.add(P.pad_kw, 1ull);
            }
            if (i < P.n) write_output<N>(P.out, nullptr, (uint64_t)i, acc.finish(P.b1));
        }
    }
}

}  // namespace pm
