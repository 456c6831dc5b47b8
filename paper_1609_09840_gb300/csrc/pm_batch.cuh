// pm_batch.cuh -- ragged batch of one-chunk strings: one persistent launch in
// which every warp works on its own tiles of WT consecutive strings.
//
// Per warp tile (claimed from a device work counter; the offsets of the
// next tile are prefetched into registers while the current one is worked):
//   plan    strings of more than one chunk (N0 > m words) go to the
//           long-string list; the bytes of the other strings are staged into
//           the warp's shared-memory slot with 1D TMA bulk copies (one per run
//           between long strings); the staged strings are partitioned by
//           length class;
//   compute a group holds 32/G strings of one length class with G = 1, 2, 4,
//           8 or 16 lanes per string, so every group takes at most 8 steps;
//           the G lanes of a string step through its words with the key words
//           from shared memory, sum their carry-free accumulators by
//           shuffles, and one lane reduces the exact sum b_1 + sum a_{1,i} s_i
//           (Sec. 5, Sec. 6.2, Alg. 2) and writes the output step.
// Each warp has two slots: the next tile's copies are in flight while the
// current tile is computed. Warps share nothing but the key.
#pragma once
#include "pm_long.cuh"

namespace pm {

constexpr int BW_WARPS = 4;                  // warps per block
constexpr int BW_THREADS = 32 * BW_WARPS;
constexpr int BW_CLASSES = 5;                // G = 1, 2, 4, 8, 16 lanes per string
// Length bins: bins 0..7 hold strings of 1..8 units (one lane each, sorted
// exactly), bins 8..11 the classes G = 2, 4, 8, 16.
constexpr int BW_BINS = 12;

// Length class of a string of `units` 8-byte units: class c holds units in
// (8 * 2^(c-1), 8 * 2^c], so G = 2^c lanes need at most 8 steps.
__device__ __forceinline__ int unit_class(uint32_t units) {
    return units <= 8 ? 0 : units <= 16 ? 1 : units <= 32 ? 2 : units <= 64 ? 3 : 4;
}

template <int WT, int DW>
struct alignas(16) WarpSlot {
    static_assert(DW < 32768, "string positions are stored as int16");
    uint8_t data[DW];                   // staged bytes (16-byte aligned)
    int16_t soff[WT];                   // string start inside data, -1 if not staged
    uint16_t len[WT];                   // string length
    uint8_t perm[WT];                   // staged strings sorted by length bin
    uint32_t hist[BW_BINS];             // strings per bin, then rank cursors
    int32_t bin_start[BW_BINS + 1];     // perm range of each bin
    int64_t s0;                         // first string of the tile
    uint64_t bar;                       // completion of the bulk copies
};

template <int N, int WT, int DW>
struct BatchWarpSmem {
    WarpSlot<WT, DW> slot[BW_WARPS][2];
    uint4 keys1[KSplit<N>::COUNT];
    uint64_t b1;
};

__device__ __forceinline__ int64_t align16_down(int64_t x) { return x & ~(int64_t)15; }
__device__ __forceinline__ int64_t align16_up(int64_t x) { return (x + 15) & ~(int64_t)15; }

// Strings the tile kernel does not hash go to the segment kernel.
template <int N>
__device__ __forceinline__ void push_long(const BatchParams &P, bool flag, int64_t string, uint64_t len) {
    reserve_segments<N>(P, flag, string, len);
}

// Offsets of one warp tile: lane l holds offsets[s0 + l + 32 e], e = 0..E.
template <int WT>
struct WarpOffs {
    static constexpr int E = WT / 32;
    int64_t v[E + 1];
};

template <int WT>
__device__ __forceinline__ void load_warp_offs(const BatchParams &P, int64_t tile, WarpOffs<WT> &o) {
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int e = 0; e <= WarpOffs<WT>::E; ++e) {
        const int64_t k = tile * WT + lane + 32 * e;
        o.v[e] = k <= P.n ? __ldg(P.off + k) : 0;
    }
}


__device__ __forceinline__ int unit_bin(uint32_t units) {
    return units <= 8 ? (int)units - 1 : 7 + unit_class(units);
}

// The last unit of a string of `len` bytes at p: its len % 8 string bytes,
// then the 0x01 pad byte of Sec. 4 (just the pad when len % 8 == 0).
__device__ __forceinline__ uint64_t smem_tail_unit(const uint8_t *p, uint32_t len) {
    const uint32_t full = len >> 3, rem = len & 7;
    uint64_t x = 0;
    if (rem) x = *reinterpret_cast<const uint64_t *>(p + 8 * full) & ((1ull << (8 * rem)) - 1);
    return x | (1ull << (8 * rem));
}

// Plan of one warp tile: long strings to the long list, staging copies,
// per-string slot position and length, and the sort by length bin.
template <int N, int WT, int DW>
__device__ __forceinline__ void warp_plan(const BatchParams &P, WarpSlot<WT, DW> &Sl, int64_t tile,
                                          const WarpOffs<WT> &o) {
    constexpr int E = WarpOffs<WT>::E;
    const int lane = threadIdx.x & 31;
    const int64_t s0 = tile * WT;
    const int cnt = (int)(P.n - s0 < WT ? P.n - s0 : WT);
    int64_t en[E];
    bool isl[E];
    unsigned lmask[E];
    bool any_long = false;
#pragma unroll
    for (int e = 0; e < E; ++e) {
        const int k = lane + 32 * e;
        const int64_t nxt = __shfl_sync(0xffffffffu, o.v[e], (lane + 1) & 31);
        const int64_t nxt0 = __shfl_sync(0xffffffffu, o.v[e + 1], 0);
        en[e] = lane < 31 ? nxt : nxt0;  // offsets[s0 + k + 1]
        const int64_t st = (o.v[e] + 7) & ~(int64_t)7;
        isl[e] = k < cnt && en[e] > st && (uint64_t)(en[e] - st) / Fam<N>::W + 1 > (uint64_t)M;
        lmask[e] = __ballot_sync(0xffffffffu, isl[e]);
        any_long |= lmask[e] != 0;
        push_long<N>(P, isl[e], s0 + k, isl[e] ? (uint64_t)(en[e] - st) : 0);
    }
    for (int b = lane; b < BW_BINS; b += 32) Sl.hist[b] = 0;
    const int64_t R0 = align16_down((__shfl_sync(0xffffffffu, o.v[0], 0) + 7) & ~(int64_t)7);
    int64_t endv = 0;  // offsets[s0 + cnt]: lane cnt%32 at e = cnt/32
#pragma unroll
    for (int e = 0; e <= E; ++e)
        if (e == cnt / 32) endv = o.v[e];
    const int64_t Rend = align16_up(__shfl_sync(0xffffffffu, endv, cnt & 31));
    bool staged[E];
    uint32_t len32[E];
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    __syncwarp();
    if (!any_long) {
        // common case: the tile spans at most WT * 1031 bytes; 32-bit positions
        const uint32_t base32 = (uint32_t)R0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = lane + 32 * e;
            const uint32_t st = ((uint32_t)o.v[e] + 7u) & ~7u;
            const uint32_t so = st - base32;
            const uint32_t l = k < cnt && (int64_t)en[e] > (int64_t)((o.v[e] + 7) & ~(int64_t)7)
                                   ? (uint32_t)en[e] - st : 0u;
            staged[e] = k < cnt && so + l <= (uint32_t)DW;
            len32[e] = l;
            Sl.soff[k] = staged[e] ? (int16_t)so : (int16_t)-1;
            Sl.len[k] = (uint16_t)(staged[e] ? l : 0);
            push_long<N>(P, k < cnt && !staged[e], s0 + k, l);  // the tile overflows the slot
        }
        if (lane == 0) {
            int64_t bytes = Rend - R0;
            if (bytes > DW) bytes = DW;
            if (bytes > 0) {
                mbar_expect_tx(&Sl.bar, (uint32_t)bytes);
                bulk_load(Sl.data, P.base + R0, (uint32_t)bytes, &Sl.bar);
            }
        }
    } else {
        // the bytes [ga, gb) inside each long string are not staged; the
        // runs between them are copied one after the other
        int64_t st[E], ga[E], gb[E], gincl[E];
        int64_t gaps = 0;
#pragma unroll
        for (int e = 0; e < E; ++e) {
            st[e] = (o.v[e] + 7) & ~(int64_t)7;
            ga[e] = align16_up(st[e]);
            gb[e] = align16_down((en[e] + 7) & ~(int64_t)7);
            if (gb[e] < ga[e]) gb[e] = ga[e];
            const int64_t gl = isl[e] ? gb[e] - ga[e] : 0;
            int64_t x = gl;
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int64_t y = __shfl_up_sync(0xffffffffu, x, d);
                if (lane >= d) x += y;
            }
            gincl[e] = gaps + x;
            gaps += __shfl_sync(0xffffffffu, x, 31);
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = lane + 32 * e;
            const int64_t gl = isl[e] ? gb[e] - ga[e] : 0;
            const int64_t l = k < cnt && en[e] > st[e] ? en[e] - st[e] : 0;
            const int64_t so = st[e] - R0 - (gincl[e] - gl);
            staged[e] = k < cnt && !isl[e] && so + l <= DW;
            len32[e] = staged[e] ? (uint32_t)l : 0u;
            Sl.soff[k] = staged[e] ? (int16_t)so : (int16_t)-1;
            Sl.len[k] = (uint16_t)len32[e];
            push_long<N>(P, k < cnt && !isl[e] && !staged[e], s0 + k, (uint64_t)l);
        }
        auto ga_of = [&](int k) -> int64_t {  // ga of string k, from its lane
            int64_t v = 0;
#pragma unroll
            for (int e = 0; e < E; ++e) {
                const int64_t x = __shfl_sync(0xffffffffu, ga[e], k & 31);
                if (e == k / 32) v = x;
            }
            return v;
        };
        auto next_long_after = [&](int k) -> int {  // first long string index > k, or WT
            int r = WT;
#pragma unroll
            for (int e = E - 1; e >= 0; --e) {
                const unsigned m = e * 32 > k ? lmask[e]
                                   : (e * 32 + 31 > k ? lmask[e] & ~((2u << (k & 31)) - 1) : 0u);
                if (m) r = e * 32 + __ffs(m) - 1;
            }
            return r;
        };
        const int first_long = next_long_after(-1);
        const int64_t run0_end = ga_of(first_long < WT ? first_long : 0);
        if (lane == 0) {
            int64_t bytes = (first_long < WT ? run0_end : Rend) - R0;
            if (bytes > DW) bytes = DW;
            if (bytes > 0) {
                mbar_expect_tx(&Sl.bar, (uint32_t)bytes);
                bulk_load(Sl.data, P.base + R0, (uint32_t)bytes, &Sl.bar);
            }
        }
#pragma unroll
        for (int e = 0; e < E; ++e) {
            const int k = lane + 32 * e;
            const int nk = next_long_after(k);
            const int64_t src1n = ga_of(nk < WT ? nk : 0);
            if (isl[e]) {
                const int64_t src0 = gb[e];
                const int64_t src1 = nk < WT ? src1n : Rend;
                const int64_t dst = gb[e] - R0 - gincl[e];
                int64_t bytes = src1 - src0;
                if (dst >= DW) bytes = 0;
                if (bytes > DW - dst) bytes = DW - dst;
                if (bytes > 0) {
                    mbar_expect_tx(&Sl.bar, (uint32_t)bytes);
                    bulk_load(Sl.data + dst, P.base + src0, (uint32_t)bytes, &Sl.bar);
                }
            }
        }
    }
    // sort the staged strings by length bin: ranks from warp-aggregated
    // shared-memory counters, then the bins' exclusive prefix
    __syncwarp();
    int bin[E];
    uint32_t rank[E];
#pragma unroll
    for (int e = 0; e < E; ++e) {
        bin[e] = staged[e] ? unit_bin(len32[e] / 8 + 1) : BW_BINS;
        const unsigned peers = __match_any_sync(0xffffffffu, bin[e]);
        const int leader = __ffs(peers) - 1;
        uint32_t b0 = 0;
        if (lane == leader && bin[e] < BW_BINS) b0 = atomicAdd(&Sl.hist[bin[e]], (uint32_t)__popc(peers));
        rank[e] = __shfl_sync(0xffffffffu, b0, leader) + __popc(peers & lanemask_lt());
    }
    __syncwarp();
    {
        const uint32_t v = lane < BW_BINS ? Sl.hist[lane] : 0;
        uint32_t x = v;
#pragma unroll
        for (int d = 1; d < 16; d <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, x, d);
            if (lane >= d) x += y;
        }
        if (lane <= BW_BINS) Sl.bin_start[lane] = (int32_t)(x - v);
        if (lane == 0) Sl.s0 = s0;
    }
    __syncwarp();
#pragma unroll
    for (int e = 0; e < E; ++e)
        if (staged[e]) Sl.perm[Sl.bin_start[bin[e]] + rank[e]] = (uint8_t)(lane + 32 * e);
    __syncwarp();
    if (lane == 0) mbar_arrive(&Sl.bar);  // after every expect_tx and slot write
}

// Sum of the full 8-byte units of a group's strings, G lanes per string.
template <int COUNT, typename Acc>
__device__ __forceinline__ void group_units(Acc &acc, const uint4 *keys1, const uint8_t *p,
                                            uint32_t full, uint32_t steps, int c, int q) {
    for (uint32_t it = 0; it < steps; ++it) {
        const uint32_t u = (it << c) + q;
        const uint4 kk = keys1[u < (uint32_t)COUNT ? u : 0];
        if (u < full) add_unit(acc, kk, *reinterpret_cast<const uint64_t *>(p + 8 * u));
    }
}

template <int N, int WT, int DW>
__device__ __forceinline__ void warp_compute(const BatchParams &P, const WarpSlot<WT, DW> &Sl,
                                             const uint4 *keys1, uint64_t b1) {
    typedef typename AccT<N>::t Acc;
    const int lane = threadIdx.x & 31;
    const int64_t s0 = Sl.s0;
    // strings of 1..8 units, sorted: one lane each
    const int n1 = Sl.bin_start[8];
#pragma unroll 1
    for (int start = 0; start < n1; start += 32) {
        const bool valid = start + lane < n1;
        const int k = valid ? Sl.perm[start + lane] : 0;
        const uint32_t len = valid ? Sl.len[k] : 0;
        const uint8_t *p = Sl.data + (valid ? Sl.soff[k] : 0);
        const uint32_t full = len >> 3;
        const uint32_t maxfull = __reduce_max_sync(0xffffffffu, full);
        Acc acc;
        acc.zero();
        group_units<KSplit<N>::COUNT>(acc, keys1, p, full, maxfull, 0, 0);
        if (valid) {
            add_unit(acc, keys1[full], smem_tail_unit(p, len));
            store_result<N>(P, s0 + k, acc.finish(b1));
        }
    }
    // longer strings: G = 2^c lanes each
#pragma unroll 1
    for (int c = 1; c < BW_CLASSES; ++c) {
        const int G = 1 << c, per = 32 >> c;
        const int s = lane >> c, q = lane & (G - 1);
        const int cend = Sl.bin_start[8 + c];
#pragma unroll 1
        for (int start = Sl.bin_start[7 + c]; start < cend; start += per) {
            const bool valid = start + s < cend;
            const int k = valid ? Sl.perm[start + s] : 0;
            const uint32_t len = valid ? Sl.len[k] : 0;
            const uint8_t *p = Sl.data + (valid ? Sl.soff[k] : 0);
            const uint32_t full = len >> 3;
            const uint32_t maxfull = __reduce_max_sync(0xffffffffu, full);
            Acc acc;
            acc.zero();
            group_units<KSplit<N>::COUNT>(acc, keys1, p, full, (maxfull + G - 1) >> c, c, q);
            for (int d = G >> 1; d > 0; d >>= 1) acc_xor_add(acc, d);
            if (valid && q == 0) {
                add_unit(acc, keys1[full], smem_tail_unit(p, len));
                store_result<N>(P, s0 + k, acc.finish(b1));
            }
        }
    }
}

template <int N, int WT, int DW>
__global__ void __launch_bounds__(BW_THREADS, 5) k_batch_warp(const BatchParams P) {
    typedef BatchWarpSmem<N, WT, DW> L;
    typedef typename Fam<N>::word word;
    extern __shared__ uint8_t smem_raw[];
    L &S = *reinterpret_cast<L *>((reinterpret_cast<uintptr_t>(smem_raw) + 127) & ~(uintptr_t)127);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const word *gkey = static_cast<const word *>(P.key);
    for (int i = tid; i < KSplit<N>::COUNT; i += BW_THREADS) S.keys1[i] = split_group<N>(gkey + 1, i);
    if (tid == 0) {
        S.b1 = (uint64_t)gkey[0];
        for (int w = 0; w < BW_WARPS; ++w) {
            mbar_init(&S.slot[w][0].bar, 1);
            mbar_init(&S.slot[w][1].bar, 1);
        }
        fence_barrier_init();
    }
    __syncthreads();
    const int64_t ntiles = (P.n + WT - 1) / WT;
    volatile int no_abort = 0;
    WarpSlot<WT, DW> *slots = S.slot[warp];
    auto claim = [&]() -> int64_t {
        int64_t t = 0;
        if (lane == 0) t = (int64_t)atomicAdd(P.tile_ctr, 1ull);
        return __shfl_sync(0xffffffffu, t, 0);
    };
    uint32_t phase[2] = {0, 0};
    int cur = 0;
    int64_t t = claim();
    WarpOffs<WT> o;
    if (t < ntiles) {
        load_warp_offs<WT>(P, t, o);
        warp_plan<N, WT, DW>(P, slots[cur], t, o);
    }
    int64_t tn = t < ntiles ? claim() : ntiles;
    if (tn < ntiles) load_warp_offs<WT>(P, tn, o);
    while (t < ntiles) {
        const int64_t tnn = tn < ntiles ? claim() : ntiles;
        WarpOffs<WT> on;
        if (tnn < ntiles) load_warp_offs<WT>(P, tnn, on);  // lands during this iteration
        if (tn < ntiles) warp_plan<N, WT, DW>(P, slots[cur ^ 1], tn, o);
        mbar_wait(&slots[cur].bar, phase[cur], &no_abort);
        phase[cur] ^= 1;
        warp_compute<N, WT, DW>(P, slots[cur], S.keys1, S.b1);
        __syncwarp();
        cur ^= 1;
        t = tn;
        tn = tnn;
        if (tn < ntiles) o = on;
    }
}

}  // namespace pm
