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
// every load instruction of a warp reads consecutive keys; one for keys of
// 6..9 units read by 16-byte loads), their loads issued before the
// multiply-adds: one short key per thread leaves too few bytes in flight to
// cover the memory latency. All threads walk the same unit
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
    // a_1, a_2; n = 64: a_1); for these and k_fixed_few, c = b_1 + the key
    // word that weighs the pad word when len % 8 == 0 (the unit after the key
    // is the word 1), c_lo + 2^64 c_hi
    uint64_t a0, a1, c_lo, c_hi;
    // keys of 2..FIXED_FEW_MAX units (k_fixed_few): the key words of units
    // 0..FIXED_FEW_MAX-1 (n = 32: a_{2u+1} | a_{2u+2} << 32; n = 64: a_{u+1})
    // and, when len % 8 == 0, the key word that weighs the pad word 1 (else
    // 0), also folded into c as above
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

// A carry-chain accumulator that starts at c = c_lo + 2^64 c_hi (b_1 plus,
// when the key's last unit is the pad word 1, that word's key word: its
// product is the key word itself), so that neither needs an add of its own.
__device__ __forceinline__ void acc_start(AccC32 &a, const FixedParams &P) {  // c < 2^33
    a.r0 = (uint32_t)P.c_lo;
    a.r1 = (uint32_t)(P.c_lo >> 32);
    a.r2 = 0;
}
__device__ __forceinline__ void acc_start(AccC64 &a, const FixedParams &P) {  // c < 2^65
    a.r0 = (uint32_t)P.c_lo;
    a.r1 = (uint32_t)(P.c_lo >> 32);
    a.r2 = (uint32_t)P.c_hi;
    a.r3 = a.r4 = 0;
    a.x0 = a.x1 = a.x2 = 0;
}
// The accumulated sum mod p (Sec. 6.2, Alg. 2): for n = 64 the cross terms
// are added in at their 32-bit shift first.
__device__ __forceinline__ Val acc_value(const AccC32 &a) { return reduce32_limbs(a.r0, a.r1, a.r2); }
__device__ __forceinline__ Val acc_value(const AccC64 &a) {
    uint32_t t[5] = {a.r0, a.r1, a.r2, a.r3, a.r4};
    add_limbs5(t, 0, a.x0, a.x1, a.x2, 0);
    return reduce64_limbs(t[0], t[1], t[2], t[3], t[4]);
}

// (c + sum of the key words times the words of the one unit x) mod p for a
// key of at most 8 bytes: one carry-chain multiply-add per word (the
// explicit 64-bit adds and compares of an earlier form cost 20% and 15% more
// time), then Sec. 6.2 and Alg. 2.
__device__ __forceinline__ Val one_unit_value(const FixedParams &P, uint64_t x, Fam<32>) {
    AccC32 acc;
    acc_start(acc, P);
    acc.add((uint32_t)P.a0, (uint32_t)x);
    acc.add((uint32_t)P.a1, (uint32_t)(x >> 32));
    return acc_value(acc);
}
__device__ __forceinline__ Val one_unit_value(const FixedParams &P, uint64_t x, Fam<64>) {
    AccC64 acc;
    acc_start(acc, P);
    acc.add(P.a0, x);
    return acc_value(acc);
}

// Keys of at most 8 bytes: the unit holds the key's bytes and, when len < 8,
// the 0x01 pad of Sec. 4; when len == 8 the pad is the next unit, the word 1,
// whose product is the constant folded into c. Two keys per thread (i,
// i + T), their loads issued together (one, four and eight keys, and two
// adjacent keys in one 16-byte load, measured slower); a 0-byte key reads
// nothing.
template <int N>
__global__ void __launch_bounds__(256) k_fixed_one(const __grid_constant__ FixedParams P) {
    typedef typename Fam<N>::word word;
    constexpr int K = 2;
    const uint32_t len = P.len;
    const uint64_t padbit = len < 8 ? 1ull << (8 * len) : 0ull;
    const uint64_t mask = len < 8 ? padbit - 1 : ~0ull;
    const uint64_t T = (uint64_t)gridDim.x * blockDim.x, n = (uint64_t)P.n;
    uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    // keys i and i + T, and their outputs, advanced by K T keys a step
    const uint64_t dk = T * P.stride;
    const uint8_t *pk = P.base + i * P.stride;
    word *po = static_cast<word *>(P.out) + i;
    for (; i < n; i += K * T, pk += K * dk, po += K * T) {
        const bool two = i + T < n;
        const uint64_t x0 = len ? __ldg(reinterpret_cast<const unsigned long long *>(pk)) : 0ull;
        const uint64_t x1 = len && two ? __ldg(reinterpret_cast<const unsigned long long *>(pk + dk)) : 0ull;
        write_output<N>(po, nullptr, 0, one_unit_value(P, (x0 & mask) | padbit, Fam<N>()));
        if (two) write_output<N>(po, nullptr, T, one_unit_value(P, (x1 & mask) | padbit, Fam<N>()));
    }
}

constexpr int FIXED_FEW_MAX = 9;  // units of the longest keys of k_fixed_few (72 bytes)

// Keys of 2..U units (9..8U bytes): every unit a full product per word on
// carry chains (the key words of a unit position are launch parameters), the
// tail unit masked with the 0x01 pad of Sec. 4, or, when len % 8 == 0, the pad
// word's key word added once; then Sec. 6.2, Alg. 2 and the output step. Two
// keys per thread (i, i + T), all their loads issued first; with V16 (a
// 16-byte aligned buffer and a stride of a multiple of 64 bytes) two units
// per 16-byte load, and for 6..9 units one key per thread (the registers of
// two keys limit residency to 4 blocks per SM; measured 5-7% faster for
// 64-byte keys, and 1-14% slower without V16). FOLD: b_1 and the pad word's key word start the
// accumulator (c) instead of being added after the units; measured faster
// for 2 units at both widths (PM+64: 11%) and 3..5 units for n = 64 (8-11%),
// and 1-5% slower for the other instances, which add them at the end.
template <int N, int U, bool V16>
__global__ void __launch_bounds__(256) k_fixed_few(const __grid_constant__ FixedParams P) {
    typedef typename AccCT<N>::t AccC;
    constexpr bool FOLD = U == 2 || (N == 64 && U == 5);
    constexpr int K = U == FIXED_FEW_MAX && V16 ? 1 : 2;  // keys per thread
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
            if constexpr (FOLD)
                acc_start(acc, P);  // b_1 and, when len % 8 == 0, the pad word's key word
            else
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
            if constexpr (FOLD) {
                if (i < P.n) write_output<N>(P.out, nullptr, (uint64_t)i, acc_value(acc));
            } else {
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
}

}  // namespace pm
