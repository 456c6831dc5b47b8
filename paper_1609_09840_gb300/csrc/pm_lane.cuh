// pm_lane.cuh -- ragged batch of strings, one lane per string.
//
// Warps step through tiles of 64 consecutive strings (grid-stride); lane j
// owns strings s0 + j and s0 + 32 + j. The sum b_1 + sum a_{1,i} s_i of a one-chunk string
// is formed with carry-free split-key multiply-adds on its 8-byte units,
// loaded straight from global memory into registers; many warps per SM hide
// the load latency (no shared-memory staging, no block barriers).
//   pass 1  every lane takes units 0..7 of its own string (the key words of
//           a position are the same for every lane: a shared-memory
//           broadcast); this finishes every string of at most 8 units;
//   pass 2  the remaining units of the tile's longer strings are cut into
//           pieces of 4 units, dealt out to the lanes 32 pieces at a time;
//           the pieces of a string (consecutive lanes) are summed by a
//           segmented shuffle reduction into its slot in shared memory,
//           which the owner lane folds in;
//   finish  the owner lane adds the tail unit (the last bytes and the 0x01
//           pad of Sec. 4), reduces (Sec. 6.2, Alg. 2) and writes the output
//           step (Sec. 5, Sec. 7): coalesced stores.
// Strings of more than one chunk are queued for the segment kernel
// (pm_long.cuh).
#pragma once
#include "pm_long.cuh"

namespace pm {

constexpr int BL_WARPS = 8;
constexpr int BL_THREADS = 32 * BL_WARPS;
constexpr int BL_PIECE = 4;  // units per pass-2 piece
constexpr int BL_SPL = 2;    // strings per lane in a tile

template <int N> struct AccWords;
template <> struct AccWords<32> { static constexpr int V = 2; };
template <> struct AccWords<64> { static constexpr int V = 6; };

template <int N>
struct LaneSmem {
    uint4 keys1[KSplit<N>::COUNT];
    uint64_t b1;
    unsigned long long part[BL_WARPS][AccWords<N>::V][32 * BL_SPL];  // pass-2 sums per string of a tile
    uint16_t pre[BL_WARPS][32 * BL_SPL + 1];                        // first pass-2 piece of each string
};

// acc += k * x for one 8-byte unit x (PTX multiply-adds: one instruction per
// 32 x 32 -> 64-bit product with a 64-bit addend).
__device__ __forceinline__ void mad_wide(uint64_t &acc, uint32_t a, uint32_t b) {
    asm("mad.wide.u32 %0, %1, %2, %0;" : "+l"(acc) : "r"(a), "r"(b));
}
__device__ __forceinline__ void mac_unit(Acc32 &acc, const uint4 &k, uint64_t x) {
    const uint32_t s0 = (uint32_t)x, s1 = (uint32_t)(x >> 32);
    mad_wide(acc.L, k.x, s0);
    mad_wide(acc.H, k.y, s0);
    mad_wide(acc.L, k.z, s1);
    mad_wide(acc.H, k.w, s1);
}
__device__ __forceinline__ void mac_unit(Acc64 &acc, const uint4 &k, uint64_t x) {
    const uint32_t s0 = (uint32_t)x, s1 = (uint32_t)(x >> 32);
    mad_wide(acc.a00, k.x, s0);
    mad_wide(acc.a01, k.x, s1);
    mad_wide(acc.a10, k.y, s0);
    mad_wide(acc.a11, k.y, s1);
    mad_wide(acc.a20, k.z, s0);
    mad_wide(acc.a21, k.z, s1);
}

// x += the value of the lane d above when that lane is in the same segment.
__device__ __forceinline__ void seg_add(Acc32 &x, int d, bool take) {
    const uint64_t L = __shfl_down_sync(0xffffffffu, x.L, d), H = __shfl_down_sync(0xffffffffu, x.H, d);
    if (take) {
        x.L += L;
        x.H += H;
    }
}
__device__ __forceinline__ void seg_add(Acc64 &x, int d, bool take) {
    const uint64_t a00 = __shfl_down_sync(0xffffffffu, x.a00, d), a01 = __shfl_down_sync(0xffffffffu, x.a01, d);
    const uint64_t a10 = __shfl_down_sync(0xffffffffu, x.a10, d), a11 = __shfl_down_sync(0xffffffffu, x.a11, d);
    const uint64_t a20 = __shfl_down_sync(0xffffffffu, x.a20, d), a21 = __shfl_down_sync(0xffffffffu, x.a21, d);
    if (take) {
        x.a00 += a00;
        x.a01 += a01;
        x.a10 += a10;
        x.a11 += a11;
        x.a20 += a20;
        x.a21 += a21;
    }
}
// part holds the accumulator words of the T strings of a tile, word c of
// string j at part[T * c + j].
template <int T>
__device__ __forceinline__ void acc_store_add(unsigned long long *part, int j, const Acc32 &a) {
    part[j] += a.L;
    part[T + j] += a.H;
}
template <int T>
__device__ __forceinline__ void acc_store_add(unsigned long long *part, int j, const Acc64 &a) {
    part[j] += a.a00;
    part[T + j] += a.a01;
    part[2 * T + j] += a.a10;
    part[3 * T + j] += a.a11;
    part[4 * T + j] += a.a20;
    part[5 * T + j] += a.a21;
}
template <int T>
__device__ __forceinline__ void acc_fold(Acc32 &a, const unsigned long long *part, int j) {
    a.L += part[j];
    a.H += part[T + j];
}
template <int T>
__device__ __forceinline__ void acc_fold(Acc64 &a, const unsigned long long *part, int j) {
    a.a00 += part[j];
    a.a01 += part[T + j];
    a.a10 += part[2 * T + j];
    a.a11 += part[3 * T + j];
    a.a20 += part[4 * T + j];
    a.a21 += part[5 * T + j];
}

// acc += the tail unit of a string of len bytes at p: its len % 8 bytes
// followed by the 0x01 pad byte of Sec. 4, at unit position len / 8.
template <typename Acc>
__device__ __forceinline__ void add_tail(Acc &acc, const uint4 *keys1, const uint8_t *p, uint32_t len) {
    const uint32_t full = len >> 3, rem = len & 7;
    const uint64_t pad = 1ull << (8 * rem);
    const uint64_t w = rem ? __ldg(reinterpret_cast<const unsigned long long *>(p) + full) : 0ull;
    mac_unit(acc, keys1[full], (w & (pad - 1)) | pad);
}

template <int N>
__global__ void __launch_bounds__(BL_THREADS, N == 32 ? 4 : 3) k_batch_lane(const BatchParams P) {
    typedef typename AccT<N>::t Acc;
    typedef typename Fam<N>::word word;
    constexpr int64_t CHUNK_BYTES = (int64_t)M * Fam<N>::W;
    constexpr int T = 32 * BL_SPL;  // strings per tile
    __shared__ LaneSmem<N> S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const word *gkey = static_cast<const word *>(P.key);
    for (int i = tid; i < KSplit<N>::COUNT; i += BL_THREADS) S.keys1[i] = split_group<N>(gkey + 1, i);
    if (tid == 0) S.b1 = (uint64_t)gkey[0];
    __syncthreads();
    const uint64_t b1 = S.b1;
    unsigned long long *part = &S.part[warp][0][0];
    uint16_t *pre = S.pre[warp];

    const uint32_t ntiles = (uint32_t)((P.n + T - 1) / T);
    const uint32_t stride = gridDim.x * BL_WARPS;
    for (uint32_t t = blockIdx.x * BL_WARPS + warp; t < ntiles; t += stride) {
        // string h * 32 + lane of the tile, h < BL_SPL
        int64_t st[BL_SPL], l[BL_SPL];
        uint32_t len[BL_SPL], full[BL_SPL], np[BL_SPL];
        bool valid[BL_SPL], one[BL_SPL];
        Acc acc[BL_SPL];
        bool any_long = false, any_med = false;
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            const int64_t s = (int64_t)t * T + h * 32 + lane;
            valid[h] = (int64_t)s < P.n;
            st[h] = 0;
            l[h] = -1;
            if (valid[h]) {
                const int64_t o0 = __ldg(P.off + s), o1 = __ldg(P.off + s + 1);
                st[h] = (o0 + 7) & ~(int64_t)7;
                l[h] = o1 > st[h] ? o1 - st[h] : 0;
            }
            one[h] = valid[h] && l[h] < CHUNK_BYTES;  // hashed here
            len[h] = one[h] ? (uint32_t)l[h] : 0;
            full[h] = len[h] >> 3;
            np[h] = full[h] > 8 ? (full[h] - 8 + BL_PIECE - 1) / BL_PIECE : 0;
            any_long |= valid[h] && !one[h];
            any_med |= np[h] != 0;
        }
        // pass 1: units 0..7 of every string
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            const unsigned long long *pu = reinterpret_cast<const unsigned long long *>(P.base + st[h]);
            uint64_t x[8];
#pragma unroll
            for (int u = 0; u < 8; ++u) x[u] = (uint32_t)u < full[h] ? __ldg(pu + u) : 0ull;
            acc[h].zero();
#pragma unroll
            for (int u = 0; u < 8; ++u) mac_unit(acc[h], S.keys1[u], x[u]);
        }
        // strings of more than one chunk: segment work items
        if (__any_sync(0xffffffffu, any_long)) {
#pragma unroll
            for (int h = 0; h < BL_SPL; ++h)
                reserve_segments<N>(P, valid[h] && !one[h], (int64_t)t * T + h * 32 + lane, (uint64_t)l[h]);
        }
        // pass 2: units 8.. of the longer strings, in pieces
        if (__any_sync(0xffffffffu, any_med)) {
            uint32_t base = 0;  // exclusive prefix of the piece counts in string order
#pragma unroll
            for (int h = 0; h < BL_SPL; ++h) {
                uint32_t x = np[h];
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
                    if (lane >= d) x += y;
                }
                pre[h * 32 + lane] = (uint16_t)(base + x - np[h]);
                base += __shfl_sync(0xffffffffu, x, 31);
#pragma unroll
                for (int c = 0; c < AccWords<N>::V; ++c) part[T * c + h * 32 + lane] = 0;
            }
            const uint32_t total = base;
            if (lane == 0) pre[T] = (uint16_t)total;
            __syncwarp();
#pragma unroll 1
            for (uint32_t q0 = 0; q0 < total; q0 += 32) {
                const uint32_t q = q0 + lane;
                int j = 0;  // last string whose first piece is <= q
#pragma unroll
                for (int step = T / 2; step > 0; step >>= 1)
                    if (pre[j + step] <= q) j += step;
                int64_t stj = 0;
                uint32_t fj = 0;
#pragma unroll
                for (int h = 0; h < BL_SPL; ++h) {
                    const int64_t a = __shfl_sync(0xffffffffu, st[h], j & 31);
                    const uint32_t f = __shfl_sync(0xffffffffu, full[h], j & 31);
                    if ((j >> 5) == h) {
                        stj = a;
                        fj = f;
                    }
                }
                const bool act = q < total;
                const uint32_t pj0 = pre[j];
                Acc pa;
                pa.zero();
                const uint32_t u0 = 8 + (q - pj0) * BL_PIECE;
                if (act) {
                    const unsigned long long *pj = reinterpret_cast<const unsigned long long *>(P.base + stj);
                    uint64_t y[BL_PIECE];
#pragma unroll
                    for (int k = 0; k < BL_PIECE; ++k) y[k] = u0 + k < fj ? __ldg(pj + u0 + k) : 0ull;
#pragma unroll
                    for (int k = 0; k < BL_PIECE; ++k)
                        mac_unit(pa, S.keys1[(u0 + k) & (KSplit<N>::COUNT - 1)], y[k]);
                }
                // sum the pieces of each string (consecutive lanes) into its first lane
                const uint32_t pj1 = pre[j + 1];
                const uint32_t qend = pj1 < q0 + 32 ? pj1 : q0 + 32;
                const int last = act ? (int)(qend - 1 - q0) : lane;  // last lane of the segment
                const uint32_t first = pj0 > q0 ? pj0 - q0 : 0;
                const uint32_t seglen = __reduce_max_sync(0xffffffffu, act ? (uint32_t)(last - lane + 1) : 1u);
                for (int d = 1; (uint32_t)d < seglen; d <<= 1) seg_add(pa, d, lane + d <= last);
                if (act && (uint32_t)lane == first) acc_store_add<T>(part, j, pa);
                __syncwarp();
            }
#pragma unroll
            for (int h = 0; h < BL_SPL; ++h)
                if (np[h]) acc_fold<T>(acc[h], part, h * 32 + lane);
            __syncwarp();
        }
        // finish
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            add_tail(acc[h], S.keys1, P.base + st[h], len[h]);
            if (one[h]) store_result<N>(P, (int64_t)t * T + h * 32 + lane, acc[h].finish(b1));
        }
    }
}

}  // namespace pm
