// pm_long.cuh -- strings of at least BIG_CHUNKS level-1 chunks in a ragged
// batch.
//
// A string of c1 level-1 chunks is cut into segments of up to m chunks; a
// segment is exactly the children of one level-2 chunk (Algorithm 1), so
// segments are independent work items.
//   reserve_big  (called by the tile kernel for each such string) reserves
//                one work item per segment and, when the string has more than
//                one segment, the tree storage of levels >= 2;
//   k_long_chunk one block per level-2 segment, thread r on chunk r: a warp
//                streams the 128-byte slabs of its 32 chunks through a ring
//                of padded shared-memory rows with 16-byte asynchronous
//                copies dealt out so that each copy instruction covers a few
//                contiguous runs (a string that starts 8 bytes past a 16-byte
//                boundary is copied from 8 bytes before it), then each thread
//                sums its own row with carry-chain multiply-adds, the key
//                words of a slab position being a shared-memory broadcast; the block sums a_{2,r} v_r, and the
//                level-2 value either is the hash or goes to the tree
//                storage, where the block that completes the last child of a
//                node computes the node (atomic arrival counters, no
//                spin-wait) up to the root.
// The chunk kernel is launched as a programmatic dependent of the tile
// kernel: its blocks may be scheduled early and wait (griddepcontrol.wait)
// until the tile kernel's work items are complete and visible.
#pragma once
#include "pm_kernels.cuh"

namespace pm {

// Strings of at least this many level-1 chunks go to the chunk kernel (one
// thread per chunk); shorter ones are hashed by one warp of the tile kernel.
constexpr uint64_t BIG_CHUNKS = 32;

// Chunk counts of the levels of a string of `len` bytes (Algorithm 1).
template <int N>
__device__ __forceinline__ int tree_counts(uint64_t len, uint64_t *c) {
    uint64_t x = len / Fam<N>::W + 1;
    int lv = 0;
    do {
        x = (x + M - 1) / M;
        c[++lv] = x;
    } while (x > 1 && lv < LMAX);
    return lv;
}

// Byte offsets inside a string's tree storage: values of levels 2..L-1
// (16 bytes each), then arrival counters of levels 3..L (4 bytes each).
struct TreeLayout {
    uint64_t vals[LMAX + 2], ctr[LMAX + 2], bytes;
};

__device__ __forceinline__ TreeLayout tree_layout(const uint64_t *c, int levels) {
    TreeLayout t;
    uint64_t off = 0;
    for (int j = 2; j < levels; ++j) {
        t.vals[j] = off;
        off += 16 * c[j];
    }
    for (int j = 3; j <= levels; ++j) {
        t.ctr[j] = off;
        off += 4 * c[j];
    }
    t.bytes = (off + 15) & ~(uint64_t)15;
    return t;
}

// Queue strings of at least BIG_CHUNKS chunks (lanes in `mask`, whole warp,
// one string at a time): reserve one work item per level-2 segment in the
// list of the chunk kernel and, when there is more than one segment, the
// tree storage of levels >= 2, laid out as tree_layout does (values of
// levels 2..L-1, then the contiguous arrival counters of levels 3..L, zeroed
// here).
template <int N>
__device__ __forceinline__ void reserve_big(const BatchParams &P, unsigned mask, int64_t string,
                                            uint64_t length) {
    const int lane = threadIdx.x & 31;
    while (mask) {
        const int src = __ffs(mask) - 1;
        mask &= mask - 1;
        const int64_t i = __shfl_sync(0xffffffffu, string, src);
        const uint64_t len = __shfl_sync(0xffffffffu, length, src);
        const uint64_t c1 = (len / Fam<N>::W + M) / M;  // ceil((len/W + 1) / m)
        const uint64_t nseg = (c1 + M - 1) / M;          // level-2 chunks
        uint64_t vbytes = 0, cbytes = 0;
        for (uint64_t x = nseg; x > 1;) {
            const uint64_t up = (x + M - 1) / M;
            vbytes += 16 * x;
            cbytes += 4 * up;
            x = up;
        }
        const uint64_t bytes = nseg > 1 ? (vbytes + cbytes + 15) & ~(uint64_t)15 : 0;
        unsigned long long pool = 0, base = 0;
        if (lane == 0) {
            if (bytes) pool = atomicAdd(P.pool_next, (unsigned long long)bytes);
            base = atomicAdd(P.big_count, (unsigned long long)nseg);
        }
        pool = __shfl_sync(0xffffffffu, pool, 0);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (pool + bytes > P.pool_cap || base + nseg > P.big_cap) {
            // refused: mark the reserved part inside the array empty
            if (lane == 0) record_status(P.status, STATUS_SCRATCH);
            for (uint64_t s = base + lane; s < P.big_cap && s < base + nseg; s += 32) P.big_str[s] = -1;
            continue;
        }
        unsigned *ctr = reinterpret_cast<unsigned *>(P.pool + pool + vbytes);
        for (uint64_t q = lane; q < cbytes / 4; q += 32) ctr[q] = 0;
        for (uint64_t s = lane; s < nseg; s += 32) {
            P.big_str[base + s] = i;
            P.big_seg[base + s] = (int32_t)s;
            P.big_pool[base + s] = bytes ? (int64_t)pool : -1;
        }
    }
}

// Levels >= 3 of a string whose level-2 chunk `seg` has value w (in lane 0):
// store it; the warp that completes the last child of a node computes the
// node, up to the root, whose value is the hash. Whole warp.
template <int N>
__device__ __forceinline__ void tree_climb(const BatchParams &P, const typename Fam<N>::word *keys, int64_t i,
                                           uint64_t seg, int64_t pool, const uint64_t *c, int levels, Val w) {
    const int lane = threadIdx.x & 31;
    const BatchParams &L = P;
    const TreeLayout tl = tree_layout(c, levels);
    uint8_t *tree = L.pool + pool;
    int j = 2;
    uint64_t node = seg;
    for (;;) {
        const uint64_t q = node / M;
        unsigned last = 0;
        if (lane == 0) {
            reinterpret_cast<Val *>(tree + tl.vals[j])[node] = w;
            __threadfence();
            const uint64_t left = c[j] - q * M;
            const unsigned expect = (unsigned)(left < (uint64_t)M ? left : (uint64_t)M);
            last = atomicAdd(reinterpret_cast<unsigned *>(tree + tl.ctr[j + 1]) + q, 1u) + 1 == expect;
        }
        if (!__shfl_sync(0xffffffffu, last, 0)) break;
        __threadfence();
        U192 pr = {0, 0, 0};
#pragma unroll
        for (int k = 0; k < M / 32; ++k) {
            const uint64_t idx = q * M + lane + 32 * k;
            if (idx < c[j]) {
                const Val *vp = reinterpret_cast<const Val *>(tree + tl.vals[j]) + idx;
                Val x;
                x.lo = __ldcg(reinterpret_cast<const unsigned long long *>(&vp->lo));
                x.hi = __ldcg(reinterpret_cast<const unsigned long long *>(&vp->hi));
                mac(pr, keys[j * KEY_ROW + 1 + lane + 32 * k], x);
            }
        }
        pr = warp_sum192(pr);
        if (lane == 0) {
            add192(pr, (uint64_t)keys[j * KEY_ROW], 0, 0);
            w = reduce<N>(pr);
        }
        ++j;
        node = q;
        if (j == levels) {
            if (lane == 0) store_result<N>(P, i, w);
            break;
        }
    }
}

constexpr int LC_THREADS = M;               // thread r owns chunk r of a segment
constexpr int LC_SLAB = 128;                // bytes of a chunk per stage
constexpr int LC_PITCH = LC_SLAB + 16;      // padded rows: consecutive rows 4 banks apart
// staging depth: 2 (at most 128 registers, 4 blocks per SM) or 3 (3 blocks)
template <int S> struct ChunkStages { static constexpr int BLOCKS = S == 2 ? 4 : 3; };

template <int N, int LC_STAGES>
struct ChunkSmem {
    uint8_t stage[LC_STAGES][LC_THREADS * LC_PITCH];
    typename UnitKey<N>::t ku[M * Fam<N>::W / 8];  // a_{1,i} of the words of unit u
    U192 part[LC_THREADS / 32];
    unsigned long long item;
};

template <int N, int S>
constexpr size_t chunk_smem_bytes() {
    return sizeof(ChunkSmem<N, S>) + 16;
}

__device__ __forceinline__ void cp_async16(void *dst, const void *src) {
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;" ::"r"(smem_addr(dst)), "l"(src) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int K>
__device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;" ::"n"(K) : "memory");
}

// Slab copies of a warp's chunks: piece q = lane + 32 k is 16-byte piece
// q % NPC of chunk q / NPC (chunks of CB bytes, rows of LC_PITCH bytes).
template <int NPC, uint64_t CB>
__device__ __forceinline__ void issue_slab(uint8_t *sb, const uint8_t *gb, int lane, int nvalid) {
#pragma unroll
    for (int k = 0; k < NPC; ++k) {
        const int q = lane + 32 * k;
        const int r = q / NPC, u = q - (q / NPC) * NPC;
        if (r < nvalid) cp_async16(sb + r * LC_PITCH + 16 * u, gb + (uint64_t)r * CB + 16 * u);
    }
}

// One work item of the chunk kernel as every thread of the block sees it.
struct ChunkItem {
    int64_t i, pool;               // string (-1: no work), tree storage
    uint64_t seg, start, len;      // level-2 segment, string span
    uint64_t c0, cend, full;       // segment chunks [c0, cend); chunk `full` is the string's tail
    const uint8_t *wsrc;           // this warp's first copied byte (16-byte aligned)
    int nvalid;                    // chunks this warp copies (0..32)
    uint32_t shift;                // 8 when the string starts 8 bytes past a 16-byte boundary
};

template <int N>
__device__ __forceinline__ ChunkItem chunk_item(const BatchParams &P, uint64_t item, uint64_t nitems, int warp) {
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;
    ChunkItem it;
    it.i = item < nitems ? P.big_str[item] : -1;  // -1 also marks a refused reservation
    it.pool = -1;
    it.seg = it.start = it.len = it.c0 = it.cend = it.full = 0;
    it.wsrc = P.base;
    it.nvalid = 0;
    it.shift = 0;
    if (it.i < 0) return it;
    it.seg = (uint64_t)P.big_seg[item];
    it.pool = P.big_pool[item];
    string_span(P.off, it.i, it.start, it.len);
    const uint64_t c1 = (it.len / Fam<N>::W + M) / M;
    it.full = it.len / CB;
    it.c0 = it.seg * M;
    it.cend = it.c0 + M < c1 ? it.c0 + M : c1;
    const uint64_t fend = it.full < it.cend ? it.full : it.cend;  // end of the copied (full) chunks
    const uint64_t wfirst = it.c0 + 32 * (uint64_t)warp;
    it.nvalid = fend > wfirst ? (int)(fend - wfirst < 32 ? fend - wfirst : 32) : 0;
    it.shift = (uint32_t)(it.start & 8);
    it.wsrc = P.base + it.start - it.shift + wfirst * CB;
    return it;
}

template <int N, int LC_STAGES>
__global__ void __launch_bounds__(LC_THREADS, ChunkStages<LC_STAGES>::BLOCKS) k_long_chunk(const BatchParams P) {
    typedef typename Fam<N>::word word;
    typedef typename AccCT<N>::t Acc;
    typedef typename UnitKey<N>::t KW;
    typedef ChunkSmem<N, LC_STAGES> Sm;
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;  // chunk bytes
    constexpr int NSLAB = (int)(CB / LC_SLAB);        // slabs per chunk: 4 or 8
    static_assert(NSLAB >= LC_STAGES - 1, "copies run at most one item ahead");
    extern __shared__ uint8_t smem_raw[];
    Sm &S = *reinterpret_cast<Sm *>((reinterpret_cast<uintptr_t>(smem_raw) + 15) & ~(uintptr_t)15);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    asm volatile("griddepcontrol.wait;" ::: "memory");  // the tile kernel's items are complete
    uint64_t nitems = *((volatile unsigned long long *)P.big_count);
    if (nitems > P.big_cap) nitems = P.big_cap;  // refused reservations are not items
    if (nitems == 0) return;
    const word *gkey = static_cast<const word *>(P.key);  // levels >= 2 and the tail: from global
    for (int u = tid; u < (int)(CB / 8); u += LC_THREADS) S.ku[u] = unit_key<N>(gkey, u);
    const uint64_t b1 = (uint64_t)gkey[0];
    uint8_t *wrow = &S.stage[0][(32 * warp) * LC_PITCH];
    const uint8_t *row = &S.stage[0][tid * LC_PITCH];
    // slab sl of an item: this warp's 32 chunks, 16-byte asynchronous copies
    // dealt to the lanes chunk by chunk (a chunk that starts 8 bytes past a
    // 16-byte boundary takes 9 pieces from 8 bytes before it); stages are
    // used in the order of a running slab counter, across items
    auto issue = [&](const ChunkItem &it, int sl, uint32_t g) {
        uint8_t *sb = wrow + (g % LC_STAGES) * (LC_THREADS * LC_PITCH);
        const uint8_t *gb = it.wsrc + sl * LC_SLAB;
        if (it.shift)
            issue_slab<9, CB>(sb, gb, lane, it.nvalid);
        else
            issue_slab<8, CB>(sb, gb, lane, it.nvalid);
        cp_async_commit();
    };
    // thread 0 claims the item after the next one while the current one is
    // hashed (the claim's latency hides behind the slab copies); `give`
    // hands its value to the block
    unsigned long long ahead = 0;
    auto give = [&](unsigned long long v) -> uint64_t {
        __syncthreads();  // S.item is free again
        if (tid == 0) S.item = v;
        __syncthreads();
        return S.item;
    };
    uint64_t cur_item = give(tid == 0 ? atomicAdd(P.big_next, 1ull) : 0ull);
    ChunkItem cur = chunk_item<N>(P, cur_item, nitems, warp);
    uint64_t nxt_item = cur_item < nitems ? give(tid == 0 ? atomicAdd(P.big_next, 1ull) : 0ull) : nitems;
    ChunkItem nxt = chunk_item<N>(P, nxt_item, nitems, warp);
    uint32_t g = 0;  // running slab counter (stage = g % LC_STAGES)
#pragma unroll
    for (int sl = 0; sl < LC_STAGES - 1; ++sl) issue(cur, sl, g + sl);
    while (cur_item < nitems) {
        if (tid == 0 && nxt_item < nitems) ahead = atomicAdd(P.big_next, 1ull);
        const uint64_t ch = cur.c0 + (uint64_t)tid;
        const bool mine = cur.i >= 0 && ch < cur.cend && ch < cur.full;
        const bool has_tail = cur.i >= 0 && cur.full >= cur.c0 && cur.full < cur.cend;
        // warp 0 loads the tail chunk's units now; they are used after the slabs
        uint64_t tu[M / 32];
#pragma unroll
        for (int q = 0; q < M / 32; ++q) tu[q] = 0;
        if (has_tail && warp == 0) {
            const uint8_t *tp = P.base + cur.start + cur.full * CB;
            const uint64_t rem = cur.len - cur.full * CB;
#pragma unroll
            for (int q = 0; q < M / 32; ++q) {
                const int wi = lane + 32 * q;  // word index in the chunk
                if constexpr (N == 32)
                    tu[q] = load_unit_padded(tp, rem, (uint64_t)(wi >> 1));
                else
                    tu[q] = load_unit_padded(tp, rem, (uint64_t)wi);
            }
        }
        Acc acc;
        acc.zero();
#pragma unroll 1
        for (int sl = 0; sl < NSLAB; ++sl, ++g) {
            __syncwarp();  // every lane is done with the stage refilled next
            const int ahead = sl + LC_STAGES - 1;  // the slab issued now, maybe of the next item
            if (ahead < NSLAB)
                issue(cur, ahead, g + LC_STAGES - 1);
            else
                issue(nxt, ahead - NSLAB, g + LC_STAGES - 1);
            cp_async_wait<LC_STAGES - 1>();  // this lane's copies of slab sl have landed
            __syncwarp();                     // and every other lane's
            if (mine) {
                // 16-byte piece j of the row holds 8-byte units 2j, 2j+1 of the
                // slab (shifted rows: units 2j-1, 2j)
                const uint4 *r = reinterpret_cast<const uint4 *>(row + (g % LC_STAGES) * (LC_THREADS * LC_PITCH));
                const KW *k1 = S.ku + sl * (LC_SLAB / 8);
                auto lo = [](const uint4 &d) { return (uint64_t)d.x | ((uint64_t)d.y << 32); };
                auto hi = [](const uint4 &d) { return (uint64_t)d.z | ((uint64_t)d.w << 32); };
                if (cur.shift) {
                    add_unit_c(acc, k1[0], hi(r[0]));
#pragma unroll
                    for (int j = 1; j < LC_SLAB / 16; ++j) {
                        const uint4 d = r[j];
                        add_unit_c(acc, k1[2 * j - 1], lo(d));
                        add_unit_c(acc, k1[2 * j], hi(d));
                    }
                    add_unit_c(acc, k1[LC_SLAB / 8 - 1], lo(r[LC_SLAB / 16]));
                } else {
#pragma unroll
                    for (int j = 0; j < LC_SLAB / 16; ++j) {
                        const uint4 d = r[j];
                        add_unit_c(acc, k1[2 * j], lo(d));
                        add_unit_c(acc, k1[2 * j + 1], hi(d));
                    }
                }
            }
        }
        if (cur.i >= 0) {
            Val v = {0, 0};
            if (mine) v = acc.finish(b1);
            // level-2 sum of the segment: sum a_{2,r} v_r over its chunks
            U192 pr = {0, 0, 0};
            if (ch < cur.cend) mac(pr, gkey[KEY_ROW + 1 + tid], v);  // v = 0 for the tail chunk
            // the tail chunk (string end, pad, zeros) by warp 0, from the
            // units it loaded before the slab loop; its product joins warp 0's share
            if (has_tail && warp == 0) {
                U192 ta = {0, 0, 0};
#pragma unroll
                for (int q = 0; q < M / 32; ++q) {
                    const int wi = lane + 32 * q;  // word index in the chunk
                    Val sv = {0, 0};
                    if constexpr (N == 32)
                        sv.lo = (wi & 1) ? (tu[q] >> 32) : (tu[q] & 0xffffffffull);
                    else
                        sv.lo = tu[q];
                    mac(ta, gkey[1 + wi], sv);
                }
                ta = warp_sum192(ta);
                if (lane == 0) {
                    add192(ta, b1, 0, 0);
                    mac(pr, gkey[KEY_ROW + 1 + (cur.full - cur.c0)], reduce<N>(ta));
                }
            }
            pr = warp_sum192(pr);
            if (lane == 0) S.part[warp] = pr;
            __syncthreads();
            if (warp == 0) {
                uint64_t c[LMAX + 2] = {0};
                const int levels = tree_counts<N>(cur.len, c);
                Val w = {0, 0};
                if (lane == 0) {
                    U192 t = S.part[0];
#pragma unroll
                    for (int k = 1; k < LC_THREADS / 32; ++k) add192(t, S.part[k]);
                    add192(t, (uint64_t)gkey[KEY_ROW], 0, 0);
                    w = reduce<N>(t);
                }
                if (levels == 2) {
                    if (lane == 0) store_result<N>(P, cur.i, w);
                } else {
                    tree_climb<N>(P, gkey, cur.i, cur.seg, cur.pool, c, levels, w);
                }
            }
        }
        cur_item = nxt_item;
        cur = nxt;
        nxt_item = cur_item < nitems ? give(ahead) : nitems;
        nxt = chunk_item<N>(P, nxt_item, nitems, warp);
    }
    cp_async_wait<0>();
}

}  // namespace pm
