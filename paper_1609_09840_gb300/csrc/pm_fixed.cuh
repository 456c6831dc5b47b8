// pm_fixed.cuh -- n keys of one length at a fixed stride (hash-table keys).
//
// Key i occupies [i * stride, i * stride + len) of the key buffer; every key
// fits in one level-1 chunk (len < m W), so its hash is the chunk value
// (b_1 + sum a_{1,i} s_i) mod p (Sec. 5, eq. 2wlinear; Sec. 6.2, Alg. 2)
// followed by the output step (Sec. 5 end, Sec. 7). k_fixed_one (keys of at
// most 8 bytes): one unit, a full product per word with explicit carries and
// the pad's constant folded into b_1; k_fixed: one thread per
// key, four units per step; k_fixed_short (keys of at most four whole units):
// K keys per thread per step (i, i + T, i + 2T, ... for T threads, so that
// every load instruction of a warp reads consecutive keys), the loads of all
// of them issued before their multiply-adds, since one short key per thread
// leaves too few bytes in flight to cover the memory latency. All threads
// walk the same unit positions, so the loop is uniform (no predication, no
// second pass) and the split key words of every position are a uniform
// operand: they travel as launch parameters (constant bank). No offsets
// array is read, and outputs are stored coalesced.
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
    const uint8_t *base;  // 8-byte aligned
    uint64_t stride;      // a multiple of 8, >= len
    int64_t n;
    uint32_t len;         // < m W bytes
    void *out;            // uint32_t / uint64_t per key
};

// keys per thread for short keys: four for n = 32, two for n = 64 (whose six
// accumulators per key take three times the registers)
template <int N> __host__ __device__ constexpr int fixed_kpt() { return N == 32 ? 4 : 2; }
constexpr uint32_t FIXED_SHORT_UNITS = 4;  // keys of at most this many whole units take several per thread

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

template <int N>
__global__ void __launch_bounds__(256, 4) k_fixed_short(const __grid_constant__ FixedParams P) {
    typedef typename AccT<N>::t Acc;
    constexpr int K = fixed_kpt<N>(), S = 2;
    static_assert(S == 2, "one whole unit at most is left after the steps");
    const uint32_t full = P.len >> 3, rem = P.len & 7;
    const uint64_t pad = 1ull << (8 * rem);
    const int64_t T = (int64_t)gridDim.x * blockDim.x;
    for (int64_t i0 = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i0 < P.n; i0 += K * T) {
        // keys i0 + j T; a key past the end reads key i0 again and stores nothing
        const unsigned long long *pk[K];
        Acc acc[K];
#pragma unroll
        for (int j = 0; j < K; ++j) {
            const int64_t i = i0 + j * T < P.n ? i0 + j * T : i0;
            pk[j] = reinterpret_cast<const unsigned long long *>(P.base + (uint64_t)i * P.stride);
            acc[j].zero();
        }
        uint32_t u = 0;
        // S units of every key per step: the loads of a step are issued together
        for (; u + S <= full; u += S) {
            uint64_t x[K][S];
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int q = 0; q < S; ++q) x[j][q] = __ldg(pk[j] + u + q);
#pragma unroll
            for (int j = 0; j < K; ++j)
#pragma unroll
                for (int q = 0; q < S; ++q) mac_unit(acc[j], P.k1[u + q], x[j][q]);
        }
        // the last whole unit (an odd count; S = 2) and the tail unit: the
        // last len % 8 bytes and the 0x01 pad of Sec. 4, loaded together
        uint64_t y[K], w[K];
        const bool odd = u < full;
#pragma unroll
        for (int j = 0; j < K; ++j) {
            y[j] = odd ? __ldg(pk[j] + u) : 0ull;
            w[j] = rem ? __ldg(pk[j] + full) : 0ull;
        }
#pragma unroll
        for (int j = 0; j < K; ++j) {
            if (odd) mac_unit(acc[j], P.k1[u], y[j]);
            if (rem)
                mac_unit(acc[j], P.k1[full], (w[j] & (pad - 1)) | pad);
            else
                add_pad_unit(acc[j], P.k1[full]);  // the unit is the word 1: its key word alone
            if (i0 + j * T < P.n) write_output<N>(P.out, nullptr, (uint64_t)(i0 + j * T), acc[j].finish(P.b1));
        }
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

}  // namespace pm
