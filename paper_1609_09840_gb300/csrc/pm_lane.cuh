// pm_lane.cuh -- ragged batch of strings, one lane per string.
//
// Warps step through tiles of 64 consecutive strings claimed from a device
// counter (a warp that meets long strings takes fewer tiles; each warp claims
// its next tile and prefetches that tile's offsets into L2 one tile ahead);
// lane j owns strings s0 + j and s0 + 32 + j of a tile. The sum
// b_1 + sum a_{1,i} s_i of a one-chunk string (Sec. 5, eq. 2wlinear) is
// formed with carry-free split-key multiply-adds on its 8-byte units, loaded
// straight from global memory into registers; many warps per SM hide the load
// latency (no shared-memory staging, no block barriers):
//   pass 1  every lane takes units 0..P1-1 of its strings (the key words
//           of a position are the same for every lane: launch parameters,
//           read from the constant bank);
//   pass 2  the remaining units of the tile's longer one-chunk strings are cut
//           into pieces of 4 units, dealt out to the lanes 32 pieces at a
//           time; the pieces of a string (consecutive lanes, each piece's
//           sum first made exact on three words for n = 64) are summed by a
//           segmented shuffle reduction into its slot in shared memory, which
//           the owner lane folds in at the finish;
//   finish  the owner lane adds the tail unit (the last bytes and the 0x01
//           pad of Sec. 4), reduces (Sec. 6.2, Alg. 2) and writes the output
//           step (Sec. 5, Sec. 7): coalesced stores.
// Strings of 2..BIG_CHUNKS-1 chunks are hashed by the whole warp right after
// the tile (hash_medium: two levels of Algorithm 1, the level-2 chunk being
// the root). Strings of BIG_CHUNKS chunks or more are queued for the chunk
// kernel (pm_long.cuh), which is launched as a programmatic dependent of this
// kernel.
#pragma once
#include "pm_long.cuh"

namespace pm {

constexpr int BL_WARPS = 8;
constexpr int BL_THREADS = 32 * BL_WARPS;
constexpr int BL_PIECE = 4;        // units per pass-2 piece
constexpr int BL_SPL = 2;          // strings per lane in a tile
constexpr int BL_T = 32 * BL_SPL;  // strings per tile

// The exact sum of one pass-2 piece as it is shuffled and stored: the two
// carry-free accumulators for n = 32, the three-word sum for n = 64 (half
// the words of its six accumulators).
template <int N> struct Piece;
template <> struct Piece<32> { typedef Acc32 t; static constexpr int V = 2; };
template <> struct Piece<64> { typedef U192 t; static constexpr int V = 3; };
__device__ __forceinline__ Acc32 to_piece(const Acc32 &a) { return a; }
__device__ __forceinline__ U192 to_piece(const Acc64 &a) { return a.total(0); }



template <int N>
struct LaneSmem {
    uint4 keys1[KSplit<N>::COUNT];                                  // level-1 keys, split
    typename Fam<N>::word keys2[KEY_ROW];                           // b_2, a_{2,1..m}
    uint64_t b1;
    unsigned long long part[BL_WARPS][Piece<N>::V][BL_T];           // pass-2 sums per string of a tile
    uint16_t pre[BL_WARPS][BL_T + 1];                               // first pass-2 piece of each string
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

// What a lane keeps of its string's pass-1 sum until the finish: the
// accumulators for n = 32, the exact three-word sum for n = 64 (fewer live
// registers through pass 2).
template <int N> struct Held;
template <> struct Held<32> { typedef Acc32 t; };
template <> struct Held<64> { typedef U192 t; };
__device__ __forceinline__ Acc32 hold(const Acc32 &a) { return a; }
__device__ __forceinline__ U192 hold(const Acc64 &a) { return a.total(0); }
// held += a * x for the tail unit x of a string, k the split key words of
// its position (n = 64: the word a = k.x + 2^25 k.y + 2^50 k.z).
__device__ __forceinline__ void add_tail_unit(Acc32 &h, const uint4 &k, uint64_t x) { mac_unit(h, k, x); }
__device__ __forceinline__ void add_tail_unit(U192 &h, const uint4 &k, uint64_t x) {
    const uint64_t a = (uint64_t)k.x | ((uint64_t)k.y << 25) | ((uint64_t)k.z << 50);
    const Val v = {x, 0};
    mac(h, a, v);
}

// x += the value of the lane d above when that lane is in the same segment.
__device__ __forceinline__ void seg_add(Acc32 &x, int d, bool take) {
    const uint64_t L = __shfl_down_sync(0xffffffffu, x.L, d), H = __shfl_down_sync(0xffffffffu, x.H, d);
    if (take) {
        x.L += L;
        x.H += H;
    }
}
__device__ __forceinline__ void seg_add(U192 &x, int d, bool take) {
    const U192 y = shfl_down192(x, d);
    if (take) add192(x, y);
}
// part holds the accumulator words of the T strings of a tile, word c of
// string j at part[T * c + j].
template <int T>
__device__ __forceinline__ void acc_store_add(unsigned long long *part, int j, const Acc32 &a) {
    part[j] += a.L;
    part[T + j] += a.H;
}
template <int T>
__device__ __forceinline__ void acc_store_add(unsigned long long *part, int j, const U192 &a) {
    U192 s = {part[j], part[T + j], part[2 * T + j]};
    add192(s, a);
    part[j] = s.w0;
    part[T + j] = s.w1;
    part[2 * T + j] = s.w2;
}
template <int T>
__device__ __forceinline__ void acc_fold(Acc32 &a, const unsigned long long *part, int j) {
    a.L += part[j];
    a.H += part[T + j];
}
// (b_1 + the string's sum) mod p: pass 1 and the tail in a, pass 2 (if any)
// in part.
template <int T>
__device__ __forceinline__ Val finish_string(const Acc32 &a, bool folded, const unsigned long long *part, int j,
                                             uint64_t b1) {
    Acc32 s = a;
    if (folded) acc_fold<T>(s, part, j);
    return s.finish(b1);
}
template <int T>
__device__ __forceinline__ Val finish_string(const U192 &a, bool folded, const unsigned long long *part, int j,
                                             uint64_t b1) {
    U192 s = a;
    add192(s, b1, 0, 0);
    if (folded) add192(s, part[j], part[T + j], part[2 * T + j]);
    return reduce<64>(s);
}

// The tail unit of a string of len bytes whose last unit (index len / 8)
// holds the word w: its len % 8 string bytes followed by the 0x01 pad byte of
// Sec. 4 (just the pad when len % 8 == 0).
__device__ __forceinline__ uint64_t tail_unit(uint64_t w, uint32_t len) {
    const uint64_t pad = 1ull << (8 * (len & 7));
    return (w & (pad - 1)) | pad;
}

// Offsets of one tile in registers: lane l holds offsets[s0 + l + 32 h]
// (h < BL_SPL) for the indices up to tend = min(s0 + BL_T, n), and every lane
// holds offsets[s0 + BL_T] when the tile is full.
struct TileOffs {
    int64_t o[BL_SPL];
    int64_t oe;
};

__device__ __forceinline__ void load_tile_offs(const BatchParams &P, uint32_t s0, uint32_t tend, TileOffs &t) {
    const uint32_t lane = threadIdx.x & 31;
#pragma unroll
    for (int h = 0; h < BL_SPL; ++h) {
        const uint32_t k = s0 + 32 * h + lane;
        t.o[h] = k <= tend ? __ldg(P.off + k) : 0;
    }
    t.oe = tend - s0 >= (uint32_t)BL_T ? __ldg(P.off + s0 + BL_T) : 0;
}

__device__ __forceinline__ int64_t align8_up(int64_t x) { return (x + 7) & ~(int64_t)7; }

// One string of 2..BIG_CHUNKS-1 level-1 chunks at p (len bytes), whole warp:
// chunk c's value v_c = (b_1 + sum_i a_{1,i} s_{mc+i}) mod p, lane l taking
// the units l, l + 32, ... of the chunk; then h = (b_2 + sum_c a_{2,c+1} v_c)
// mod p (Algorithm 1: with at most m chunks the level-2 chunk is the root).
// The loads of chunk c + 1 are in flight while chunk c is reduced.
template <int N>
__device__ __noinline__ void hash_medium(const BatchParams &P, const LaneSmem<N> &S, int64_t i, uint64_t st,
                                         uint64_t len) {
    typedef typename AccT<N>::t Acc;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;    // units per lane per chunk: 2 or 4
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;  // chunk bytes
    const int lane = threadIdx.x & 31;
    const uint8_t *p = P.base + st;
    const uint64_t c1 = (len / Fam<N>::W + M) / M;  // ceil((len / W + 1) / m)
    const uint64_t full = len / CB;                 // chunks of string bytes only
    auto load = [&](uint64_t c, uint64_t (&x)[UPL]) {
        const uint8_t *cp = p + c * CB;
#pragma unroll
        for (int q = 0; q < UPL; ++q) {
            const uint64_t u = (uint64_t)(lane + 32 * q);
            x[q] = c < full ? __ldg(reinterpret_cast<const unsigned long long *>(cp) + u)
                            : load_unit_padded(cp, len - c * CB, u);
        }
    };
    uint64_t x[UPL], y[UPL];
    load(0, x);
    U192 s2 = {0, 0, 0};
    for (uint64_t c = 0; c < c1; ++c) {
        if (c + 1 < c1) load(c + 1, y);
        Acc a;
        a.zero();
#pragma unroll
        for (int q = 0; q < UPL; ++q) mac_unit(a, S.keys1[lane + 32 * q], x[q]);
        warp_allsum(a);
        if (lane == 0) mac(s2, S.keys2[1 + c], a.finish(S.b1));
#pragma unroll
        for (int q = 0; q < UPL; ++q) x[q] = y[q];
    }
    if (lane == 0) {
        add192(s2, (uint64_t)S.keys2[0], 0, 0);
        store_result<N>(P, i, reduce<N>(s2));
    }
}

// P1: units of every string taken by pass 1 (6 or 8, picked by the autotuner).
template <int N, int P1>
__global__ void __launch_bounds__(BL_THREADS, N == 32 ? 4 : 3) k_batch_lane(const __grid_constant__ BatchParams P) {
    typedef typename AccT<N>::t Acc;
    typedef typename Fam<N>::word word;
    static_assert(P1 <= BL_P1_MAX, "pass-1 key words travel as launch parameters");
    constexpr int64_t CHUNK_BYTES = (int64_t)M * Fam<N>::W;
    constexpr int T = BL_T;
    __shared__ LaneSmem<N> S;
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the chunk kernel, when it follows (big_cap > 0), may be scheduled now: it
    // waits for this grid's results; otherwise nothing may start early
    if (P.big_cap) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const word *gkey = static_cast<const word *>(P.key);
    for (int i = tid; i < KSplit<N>::COUNT; i += BL_THREADS) S.keys1[i] = split_group<N>(gkey + 1, i);
    for (int i = tid; i < KEY_ROW; i += BL_THREADS) S.keys2[i] = gkey[KEY_ROW + i];
    if (tid == 0) S.b1 = (uint64_t)gkey[0];
    __syncthreads();
    const uint64_t b1 = S.b1;
    unsigned long long *part = &S.part[warp][0][0];
    uint16_t *pre = S.pre[warp];

    // tiles: warp gw starts with tile gw and then claims tiles nw, nw + 1, ...
    // from a device counter, one tile ahead (string indices fit in 32 bits)
    const uint32_t n = (uint32_t)P.n;
    const uint32_t ntiles = (uint32_t)((P.n + T - 1) / T);
    const uint32_t gw = blockIdx.x * BL_WARPS + warp, nw = gridDim.x * BL_WARPS;
    if (gw >= ntiles) return;
    unsigned ticket = 0;  // claim of the next tile (lane 0)
    if (lane == 0) ticket = atomicAdd(P.tile_ctr, 1u);
    for (uint32_t t = gw; t < ntiles;) {
        const uint32_t s0 = t * T;
        const uint32_t tend = n - s0 < (uint32_t)T ? n : s0 + T;
        const int cnt = (int)(tend - s0);
        TileOffs cur;
        load_tile_offs(P, s0, tend, cur);
        // the next tile: claimed a tile ago; prefetch its offsets, claim the one after
        const uint32_t tn = nw + __shfl_sync(0xffffffffu, ticket, 0);
        if (tn < ntiles) {
            const uint32_t k = tn * T + 16 * lane;  // one 128-byte line of offsets per lane
            if (lane <= T / 16 && k <= n) prefetch_l2(P.off + k);
            if (lane == 0) ticket = atomicAdd(P.tile_ctr, 1u);
        }
        // string h * 32 + lane of the tile, h < BL_SPL
        int64_t st[BL_SPL];
        uint32_t len[BL_SPL], full[BL_SPL];
        bool one[BL_SPL], med[BL_SPL];
        bool any_med = false;
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            const int64_t nx = __shfl_sync(0xffffffffu, cur.o[h], (lane + 1) & 31);
            const int64_t n0 = __shfl_sync(0xffffffffu, cur.o[h + 1 < BL_SPL ? h + 1 : 0], 0);
            const int64_t e = lane < 31 ? nx : (h + 1 < BL_SPL ? n0 : cur.oe);
            const bool valid = 32 * h + lane < cnt;
            st[h] = align8_up(cur.o[h]);
            const int64_t l = valid ? (e > st[h] ? e - st[h] : 0) : -1;
            one[h] = valid && l < CHUNK_BYTES;  // hashed by the lane
            const bool longer = valid && !one[h];
            const bool big = longer && (uint64_t)l / Fam<N>::W + 1 > (uint64_t)M * (BIG_CHUNKS - 1);
            // strings of at least BIG_CHUNKS chunks: work items of the chunk kernel
            const unsigned bb = __ballot_sync(0xffffffffu, big);
            if (bb) reserve_big<N>(P, bb, (int64_t)(s0 + 32 * h + lane), big ? (uint64_t)l : 0);
            med[h] = longer && !big;  // hashed by the whole warp
            len[h] = one[h] ? (uint32_t)l : 0u;
            full[h] = len[h] >> 3;
            any_med |= full[h] > P1;
        }
        // pass 1: units 0..P1-1 of every one-chunk string
        typename Held<N>::t acc[BL_SPL];
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            const unsigned long long *pu = reinterpret_cast<const unsigned long long *>(P.base + st[h]);
            uint64_t x[P1];
#pragma unroll
            for (int u = 0; u < P1; ++u) x[u] = (uint32_t)u < full[h] ? __ldg(pu + u) : 0ull;
            Acc a1;
            a1.zero();
#pragma unroll
            for (int u = 0; u < P1; ++u) mac_unit(a1, P.k1[u], x[u]);  // key words: launch parameters
            acc[h] = hold(a1);
        }
        // pass 2: units 8.. of the longer one-chunk strings, in pieces
        if (__any_sync(0xffffffffu, any_med)) {
            uint32_t np[BL_SPL];  // pieces of each string
#pragma unroll
            for (int h = 0; h < BL_SPL; ++h)
                np[h] = full[h] > P1 ? (full[h] - P1 + BL_PIECE - 1) / BL_PIECE : 0;
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
                for (int c = 0; c < Piece<N>::V; ++c) part[T * c + h * 32 + lane] = 0;
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
                const uint32_t u0 = P1 + (q - pj0) * BL_PIECE;
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
                typename Piece<N>::t ps = to_piece(pa);
                const uint32_t pj1 = pre[j + 1];
                const uint32_t qend = pj1 < q0 + 32 ? pj1 : q0 + 32;
                const int last = act ? (int)(qend - 1 - q0) : lane;  // last lane of the segment
                const uint32_t first = pj0 > q0 ? pj0 - q0 : 0;
                const uint32_t seglen = __reduce_max_sync(0xffffffffu, act ? (uint32_t)(last - lane + 1) : 1u);
                for (int d = 1; (uint32_t)d < seglen; d <<= 1) seg_add(ps, d, lane + d <= last);
                if (act && (uint32_t)lane == first) acc_store_add<T>(part, j, ps);
                __syncwarp();
            }
        }
        // finish: the tail unit (its line was just read: an L1 hit), reduction,
        // output step
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            const uint64_t tw =
                len[h] & 7 ? __ldg(reinterpret_cast<const unsigned long long *>(P.base + st[h]) + full[h]) : 0ull;
            add_tail_unit(acc[h], S.keys1[full[h]], tail_unit(tw, len[h]));
        }
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h)
            if (one[h])
                store_result<N>(P, (int64_t)(s0 + 32 * h + lane),
                                finish_string<T>(acc[h], full[h] > P1, part, h * 32 + lane, b1));
        __syncwarp();  // part[] is read before the next tile clears it
        // strings of 2..BIG_CHUNKS-1 chunks: the whole warp, one at a time
#pragma unroll
        for (int h = 0; h < BL_SPL; ++h) {
            unsigned mm = __ballot_sync(0xffffffffu, med[h]);
            while (mm) {
                const int src = __ffs(mm) - 1;
                mm &= mm - 1;
                const int64_t i = (int64_t)(s0 + 32 * h + src);
                const int64_t ms = __shfl_sync(0xffffffffu, st[h], src);
                const int64_t me = __ldg(P.off + i + 1);
                hash_medium<N>(P, S, i, (uint64_t)ms, (uint64_t)(me - ms));
            }
        }
        t = tn;
    }
}

}  // namespace pm
