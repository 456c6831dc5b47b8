// pm_lane.cuh -- ragged batch of strings, one lane per string.
//
// Every one-chunk string is hashed by one lane: its 8-byte units are loaded
// straight from global memory into registers (one predicated load per unit),
// b_1 + sum a_{1,i} s_i is formed with carry-free split-key multiply-adds
// (the key words of a position are the same for every lane of a warp: a
// shared-memory broadcast), reduced (Sec. 6.2, Alg. 2) and mixed (Sec. 5,
// Sec. 7) by the same lane.
//   k_batch_lane    warps step through sub-tiles of 32 consecutive strings
//                   (grid-stride); lane l owns string s0 + l. Short strings
//                   (at most 8 units: up to 63 bytes) are hashed at once,
//                   with coalesced stores. Medium strings (9 units up to one
//                   chunk) are sorted by unit count into three classes (9..16,
//                   17..32, 33 up to one chunk), gathered per warp in shared
//                   memory and appended 32 at a time to a global list per
//                   class. Longer strings are queued for the segment kernel
//                   (pm_long.cuh). Few registers: many warps per SM hide the
//                   load latency.
//   k_batch_medium  one lane per listed string, 32 strings of one class per
//                   warp, so that the lanes of a warp have similar lengths.
#pragma once
#include "pm_long.cuh"

namespace pm {

constexpr int BL_WARPS = 8;
constexpr int BL_THREADS = 32 * BL_WARPS;
constexpr int BL_RING = 64;   // entries of a warp's queue (a power of two)
constexpr int BL_QUEUES = 3;  // medium classes: 9..16, 17..32, 33.. units

template <int N>
struct LaneSmem {
    uint4 keys1[KSplit<N>::COUNT];
    uint64_t b1;
    uint32_t q_str[BL_WARPS][BL_QUEUES][BL_RING];  // medium strings not yet listed
};

constexpr uint32_t NOT_ONE_CHUNK = 0xffffffffu;

// acc += a * unit u of the string at p when u < full (else nothing): one
// predicated 8-byte load and the split-key multiply-adds, in PTX so that the
// predicate guards the load and the products alike. OFF is a byte offset
// added to p in the load's address.
template <int OFF = 0>
__device__ __forceinline__ void unit_if(Acc32 &acc, const uint4 &k, const void *p, uint32_t u, uint32_t full) {
    asm("{\n\t.reg .pred q;\n\t.reg .b32 s0, s1;\n\t"
        "setp.lt.u32 q, %2, %3;\n\t"
        "@q ld.global.nc.v2.u32 {s0, s1}, [%4+%9];\n\t"
        "@q mad.wide.u32 %0, %5, s0, %0;\n\t"
        "@q mad.wide.u32 %1, %6, s0, %1;\n\t"
        "@q mad.wide.u32 %0, %7, s1, %0;\n\t"
        "@q mad.wide.u32 %1, %8, s1, %1;\n\t}"
        : "+l"(acc.L), "+l"(acc.H)
        : "r"(u), "r"(full), "l"(p), "r"(k.x), "r"(k.y), "r"(k.z), "r"(k.w), "n"(OFF));
}
template <int OFF = 0>
__device__ __forceinline__ void unit_if(Acc64 &acc, const uint4 &k, const void *p, uint32_t u, uint32_t full) {
    asm("{\n\t.reg .pred q;\n\t.reg .b32 s0, s1;\n\t"
        "setp.lt.u32 q, %6, %7;\n\t"
        "@q ld.global.nc.v2.u32 {s0, s1}, [%8+%12];\n\t"
        "@q mad.wide.u32 %0, %9, s0, %0;\n\t"
        "@q mad.wide.u32 %1, %9, s1, %1;\n\t"
        "@q mad.wide.u32 %2, %10, s0, %2;\n\t"
        "@q mad.wide.u32 %3, %10, s1, %3;\n\t"
        "@q mad.wide.u32 %4, %11, s0, %4;\n\t"
        "@q mad.wide.u32 %5, %11, s1, %5;\n\t}"
        : "+l"(acc.a00), "+l"(acc.a01), "+l"(acc.a10), "+l"(acc.a11), "+l"(acc.a20), "+l"(acc.a21)
        : "r"(u), "r"(full), "l"(p), "r"(k.x), "r"(k.y), "r"(k.z), "n"(OFF));
}

// acc += the tail unit of a string of len bytes at p: its len % 8 bytes
// followed by the 0x01 pad byte of Sec. 4, at unit position len / 8.
template <typename Acc>
__device__ __forceinline__ void add_tail(Acc &acc, const uint4 *keys1, const uint8_t *p, uint32_t len) {
    const uint32_t full = len >> 3, rem = len & 7;
    const uint64_t pad = 1ull << (8 * rem);
    const uint64_t w = rem ? __ldg(reinterpret_cast<const unsigned long long *>(p) + full) : 0ull;
    add_unit(acc, keys1[full], (w & (pad - 1)) | pad);
}

// Hash one medium string per lane (len bytes at p; lanes with ok false
// take part in the loads' control flow only): units in batches of 8.
template <int N>
__device__ __forceinline__ Val lane_medium(const uint4 *keys1, uint64_t b1, const uint8_t *p, uint32_t len) {
    typedef typename AccT<N>::t Acc;
    const uint32_t full = len >> 3;
    const uint32_t umax = __reduce_max_sync(0xffffffffu, full);
    Acc acc;
    acc.zero();
#pragma unroll 1
    for (uint32_t ub = 0; ub < umax; ub += 4) {
#pragma unroll
        for (int j = 0; j < 4; ++j)
            unit_if(acc, keys1[(ub + j) & (KSplit<N>::COUNT - 1)], p + 8 * (ub + j), ub + j, full);
    }
    add_tail(acc, keys1, p, len);
    return acc.finish(b1);
}

// Append `cnt` (<= 32) queued strings of class k, from queue position
// `first`, to the global list of the class.
template <int N>
__device__ __forceinline__ void list_medium(const BatchParams &P, const LaneSmem<N> &S, int warp, int k,
                                            uint32_t first, uint32_t cnt) {
    const int lane = threadIdx.x & 31;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(P.med_count + k, (unsigned long long)cnt);
    base = __shfl_sync(0xffffffffu, base, 0);
    if ((uint32_t)lane < cnt) {
        const uint64_t idx = base + (uint64_t)lane;
        if (idx < P.med_cap[k])
            P.med_list[k][idx] = S.q_str[warp][k][(first + (uint32_t)lane) & (BL_RING - 1)];
        else
            record_status(STATUS_SCRATCH);
    }
}

template <int N>
__global__ void __launch_bounds__(BL_THREADS, N == 32 ? 5 : 4) k_batch_lane(const BatchParams P) {
    typedef typename AccT<N>::t Acc;
    typedef typename Fam<N>::word word;
    constexpr int64_t CHUNK_BYTES = (int64_t)M * Fam<N>::W;
    __shared__ LaneSmem<N> S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const word *gkey = static_cast<const word *>(P.key);
    for (int i = tid; i < KSplit<N>::COUNT; i += BL_THREADS) S.keys1[i] = split_group<N>(gkey + 1, i);
    if (tid == 0) S.b1 = (uint64_t)gkey[0];
    __syncthreads();
    const uint64_t b1 = S.b1;
    uint32_t qh[BL_QUEUES] = {0, 0, 0}, qt[BL_QUEUES] = {0, 0, 0};

    const uint32_t ntiles = (uint32_t)((P.n + 31) / 32);
    const uint32_t stride = gridDim.x * BL_WARPS;
    for (uint32_t t = blockIdx.x * BL_WARPS + warp; t < ntiles; t += stride) {
        const uint32_t s = t * 32 + lane;
        const bool valid = (int64_t)s < P.n;
        int64_t st = 0, l = -1;
        if (valid) {
            const int64_t o0 = __ldg(P.off + s), o1 = __ldg(P.off + s + 1);
            st = (o0 + 7) & ~(int64_t)7;
            l = o1 > st ? o1 - st : 0;
        }
        const uint32_t len = (uint32_t)l;  // meaningful when 0 <= l < CHUNK_BYTES
        const uint8_t *p = P.base + st;
        // short strings
        const bool shrt = valid && l < 64;
        const uint32_t full = shrt ? len >> 3 : 0;
        Acc acc;
        acc.zero();
        unit_if<0>(acc, S.keys1[0], p, 0, full);
        unit_if<8>(acc, S.keys1[1], p, 1, full);
        unit_if<16>(acc, S.keys1[2], p, 2, full);
        unit_if<24>(acc, S.keys1[3], p, 3, full);
        unit_if<32>(acc, S.keys1[4], p, 4, full);
        unit_if<40>(acc, S.keys1[5], p, 5, full);
        unit_if<48>(acc, S.keys1[6], p, 6, full);
        add_tail(acc, S.keys1, p, shrt ? len : 0);
        if (shrt) store_result<N>(P, (int64_t)s, acc.finish(b1));
        // strings of more than one chunk: segment work items
        const bool isl = valid && l >= CHUNK_BYTES;
        if (__any_sync(0xffffffffu, isl)) reserve_segments<N>(P, isl, (int64_t)s, (uint64_t)l);
        // medium strings: per-warp queues by unit count, listed 32 at a time
        const bool med = valid && l >= 64 && l < CHUNK_BYTES;
        if (__any_sync(0xffffffffu, med)) {
            const uint32_t mf = len >> 3;
            const int c = mf < 16 ? 0 : (mf < 32 ? 1 : 2);
#pragma unroll
            for (int k = 0; k < BL_QUEUES; ++k) {
                const bool f = med && c == k;
                const unsigned m = __ballot_sync(0xffffffffu, f);
                if (f) S.q_str[warp][k][(qh[k] + (uint32_t)__popc(m & lanemask_lt())) & (BL_RING - 1)] = s;
                qh[k] += (uint32_t)__popc(m);
            }
            __syncwarp();
#pragma unroll 1
            for (int k = 0; k < BL_QUEUES; ++k)
                if (qh[k] - qt[k] >= 32u) {
                    list_medium<N>(P, S, warp, k, qt[k], 32u);
                    qt[k] += 32u;
                }
            __syncwarp();
        }
    }
    // the rest of the queues
    __syncwarp();
#pragma unroll 1
    for (int k = 0; k < BL_QUEUES; ++k)
        if (qh[k] != qt[k]) list_medium<N>(P, S, warp, k, qt[k], qh[k] - qt[k]);
}

template <int N>
__global__ void __launch_bounds__(BL_THREADS) k_batch_medium(const BatchParams P) {
    typedef typename Fam<N>::word word;
    __shared__ uint4 keys1[KSplit<N>::COUNT];
    const int tid = threadIdx.x, lane = tid & 31;
    const word *gkey = static_cast<const word *>(P.key);
    for (int i = tid; i < KSplit<N>::COUNT; i += BL_THREADS) keys1[i] = split_group<N>(gkey + 1, i);
    __syncthreads();
    const uint64_t b1 = (uint64_t)gkey[0];
    uint64_t cnt[BL_QUEUES], groups[BL_QUEUES], total = 0;
#pragma unroll
    for (int k = 0; k < BL_QUEUES; ++k) {
        const uint64_t c = *((volatile unsigned long long *)P.med_count + k);
        cnt[k] = c < P.med_cap[k] ? c : P.med_cap[k];
        groups[k] = (cnt[k] + 31) / 32;
        total += groups[k];
    }
    const uint64_t stride = (uint64_t)gridDim.x * BL_WARPS;
    // longest class first
    for (uint64_t g = (uint64_t)blockIdx.x * BL_WARPS + (tid >> 5); g < total; g += stride) {
        int k = BL_QUEUES - 1;
        uint64_t j = g;
        while (j >= groups[k]) j -= groups[k--];
        const uint64_t idx = j * 32 + (uint64_t)lane;
        const bool ok = idx < cnt[k];
        int64_t st = 0;
        uint32_t len = 0;
        int64_t s = 0;
        if (ok) {
            s = (int64_t)P.med_list[k][idx];
            const int64_t o0 = __ldg(P.off + s), o1 = __ldg(P.off + s + 1);
            st = (o0 + 7) & ~(int64_t)7;
            len = (uint32_t)(o1 - st);
        }
        const Val v = lane_medium<N>(keys1, b1, P.base + st, len);
        if (ok) store_result<N>(P, s, v);
    }
}

}  // namespace pm
