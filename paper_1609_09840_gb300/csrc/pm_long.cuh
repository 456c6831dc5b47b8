// pm_long.cuh -- strings of more than one level-1 chunk in a ragged batch.
//
// A string of c1 level-1 chunks is cut into segments of up to m chunks; a
// segment is exactly the children of one level-2 chunk (Algorithm 1), so
// segments are independent work items.
//   reserve_segments  (called by the tile kernel for each string it does not
//                hash) reserves the string's segments' work items and, when it
//                has more than one segment, the tree storage of levels >= 2;
//   k_long_seg   persistent warps claim segments. A warp hashes 4 level-1
//                chunks at a time: lane l owns the same word positions of
//                every chunk (coalesced loads, level-1 key words in
//                registers), the 4 chunks' carry-free accumulators are summed
//                across lanes by one butterfly transposition (each step sends
//                half of the remaining chunks), one lane per chunk reduces
//                its exact sum (Sec. 6.2, Alg. 2) and folds a_{2,c} v_c into
//                the segment's level-2 sum. The level-2 value either is the
//                hash, or goes to the tree storage, where the warp that
//                completes the last child of a node computes the node
//                (atomic arrival counter, no spin-wait) up to the root.
#pragma once
#include "pm_kernels.cuh"

namespace pm {

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

// Queue strings of more than one segment (lanes in `mask`, whole warp, one
// string at a time): reserve the string's segment work items and its tree
// storage of levels >= 2, laid out as tree_layout does (values of levels
// 2..L-1, then the contiguous arrival counters of levels 3..L, zeroed here).
template <int N>
__device__ __forceinline__ void reserve_multi(const BatchParams &P, unsigned mask, int64_t string,
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
        const uint64_t bytes = (vbytes + cbytes + 15) & ~(uint64_t)15;
        unsigned long long pool = 0, base = 0;
        if (lane == 0) {
            pool = atomicAdd(P.pool_next, (unsigned long long)bytes);
            base = atomicAdd(P.item_count, (unsigned long long)nseg);
        }
        pool = __shfl_sync(0xffffffffu, pool, 0);
        base = __shfl_sync(0xffffffffu, base, 0);
        if (pool + bytes > P.pool_cap || base + nseg > P.item_cap) {
            // refused: mark the reserved part inside the array empty
            if (lane == 0) record_status(STATUS_SCRATCH);
            for (uint64_t s = base + lane; s < P.item_cap && s < base + nseg; s += 32) P.item_str[s] = -1;
            continue;
        }
        unsigned *ctr = reinterpret_cast<unsigned *>(P.pool + pool + vbytes);
        for (uint64_t q = lane; q < cbytes / 4; q += 32) ctr[q] = 0;
        for (uint64_t s = lane; s < nseg; s += 32) {
            P.item_str[base + s] = i;
            P.item_seg[base + s] = (int32_t)s;
            P.item_pool[base + s] = (int64_t)pool;
        }
    }
}

// Queue the flagged lanes' strings for the segment kernel (called by the
// tile kernel, whole warp, for every string it does not hash itself).
// Strings of one segment take one work item each, appended warp-aggregated;
// longer strings go through reserve_multi.
template <int N>
__device__ __forceinline__ void reserve_segments(const BatchParams &P, bool flag, int64_t string,
                                                 uint64_t length) {
    const unsigned b = __ballot_sync(0xffffffffu, flag);
    if (!b) return;
    const bool multi = flag && length / Fam<N>::W + 1 > (uint64_t)M * M;
    const unsigned bm = __ballot_sync(0xffffffffu, multi);
    const unsigned bs = b & ~bm;
    if (bs) {
        unsigned long long base = 0;
        if ((threadIdx.x & 31) == 0) base = atomicAdd(P.item_count, (unsigned long long)__popc(bs));
        base = __shfl_sync(0xffffffffu, base, 0);
        if (flag && !multi) {
            const uint64_t s = base + (uint64_t)__popc(bs & lanemask_lt());
            if (s < P.item_cap) {
                P.item_str[s] = string;
                P.item_seg[s] = 0;
                P.item_pool[s] = -1;
            } else {
                record_status(STATUS_SCRATCH);
            }
        }
    }
    if (bm) reserve_multi<N>(P, bm, string, length);
}

// Butterfly transposition of the accumulators of 4 chunks: afterwards every
// lane holds the warp total of chunk 2*bit4(lane) + bit3(lane).
__device__ __forceinline__ void xpose_add(Acc32 &a, const Acc32 &b, int d) {
    a.L += __shfl_xor_sync(0xffffffffu, b.L, d);
    a.H += __shfl_xor_sync(0xffffffffu, b.H, d);
}
__device__ __forceinline__ void xpose_add(Acc64 &a, const Acc64 &b, int d) {
    a.a00 += __shfl_xor_sync(0xffffffffu, b.a00, d);
    a.a01 += __shfl_xor_sync(0xffffffffu, b.a01, d);
    a.a10 += __shfl_xor_sync(0xffffffffu, b.a10, d);
    a.a11 += __shfl_xor_sync(0xffffffffu, b.a11, d);
    a.a20 += __shfl_xor_sync(0xffffffffu, b.a20, d);
    a.a21 += __shfl_xor_sync(0xffffffffu, b.a21, d);
}

template <typename Acc>
__device__ __forceinline__ Acc transpose4(Acc A[4]) {
    const int lane = threadIdx.x & 31;
    const bool hi4 = lane & 16, hi3 = lane & 8;
    // step 1: keep chunks {0,1} or {2,3}, receive the partner's share of them
    Acc k0 = hi4 ? A[2] : A[0], k1 = hi4 ? A[3] : A[1];
    const Acc s0 = hi4 ? A[0] : A[2], s1 = hi4 ? A[1] : A[3];
    xpose_add(k0, s0, 16);
    xpose_add(k1, s1, 16);
    // step 2: keep one of the two
    Acc k = hi3 ? k1 : k0;
    const Acc s = hi3 ? k0 : k1;
    xpose_add(k, s, 8);
    // steps 3-5: all-reduce within the 8 lanes holding the same chunk
    xpose_add(k, k, 4);
    xpose_add(k, k, 2);
    xpose_add(k, k, 1);
    return k;
}

template <int N>
__global__ void __launch_bounds__(256) k_long_seg(const BatchParams L) {
    typedef typename Fam<N>::word word;
    typedef typename AccT<N>::t Acc;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;  // 8-byte units per lane per chunk: 2 or 4
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;  // chunk bytes
    __shared__ word keys[LMAX * KEY_ROW];
    const BatchParams &P = L;
    const word *gkey = static_cast<const word *>(P.key);
    for (int t = threadIdx.x; t < LMAX * KEY_ROW; t += blockDim.x) keys[t] = gkey[t];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint4 kr[UPL];
#pragma unroll
    for (int q = 0; q < UPL; ++q) kr[q] = split_group<N>(keys + 1, lane + 32 * q);
    uint64_t nitems = *((volatile unsigned long long *)L.item_count);
    if (nitems > L.item_cap) nitems = L.item_cap;  // refused reservations are not items
    const int own_chunk = ((lane >> 4) & 1) * 2 + ((lane >> 3) & 1);  // chunk of a 4-chunk step
    // claim segments four at a time when there are many, one at a time else
    const uint64_t warps = (uint64_t)gridDim.x * (blockDim.x / 32);
    const unsigned long long grab = nitems > 16 * warps ? 4ull : 1ull;
    uint64_t claimed = 0, claim_end = 0;
    for (;;) {
        if (claimed == claim_end) {
            unsigned long long b = 0;
            if (lane == 0) b = atomicAdd(L.item_next, grab);
            b = __shfl_sync(0xffffffffu, b, 0);
            claimed = b;
            claim_end = b + grab < nitems ? b + grab : nitems;
            if (claimed >= nitems) break;
        }
        const uint64_t item = claimed++;
        const int64_t i = L.item_str[item];
        if (i < 0) continue;  // part of a refused reservation
        const uint64_t seg = (uint64_t)L.item_seg[item];
        const int64_t pool = L.item_pool[item];
        uint64_t start, len;
        string_span(P.off, i, start, len);
        const uint8_t *p = P.base + start;
        uint64_t c[LMAX + 2] = {0};
        const int levels = tree_counts<N>(len, c);
        const uint64_t c1 = c[1], full = len / CB;  // chunks of string bytes only
        const uint64_t c0 = seg * M, cend = c0 + M < c1 ? c0 + M : c1;
        // lane's units of 4 consecutive chunks (zero beyond the segment)
        auto load4 = [&](uint64_t cb, uint64_t (&x)[4][UPL]) {
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                const uint64_t ch = cb + cc;
                const uint8_t *cp = p + ch * CB;
#pragma unroll
                for (int q = 0; q < UPL; ++q) {
                    const uint64_t u = (uint64_t)(lane + 32 * q);
                    x[cc][q] = ch < full ? __ldg(reinterpret_cast<const unsigned long long *>(cp + 8 * u))
                               : ch < cend ? load_unit_padded(cp, len - ch * CB, u)
                                           : 0ull;
                }
            }
        };
        U192 s2 = {0, 0, 0};
        Val v1 = {0, 0};
        uint64_t x[4][UPL];
        load4(c0, x);
        for (uint64_t cb = c0; cb < cend; cb += 4) {
            Acc A[4];
#pragma unroll
            for (int cc = 0; cc < 4; ++cc) {
                A[cc].zero();
#pragma unroll
                for (int q = 0; q < UPL; ++q) add_unit(A[cc], kr[q], x[cc][q]);
            }
            if (cb + 4 < cend) load4(cb + 4, x);  // in flight during the reduction below
            const Acc t = transpose4(A);
            const uint64_t ch = cb + own_chunk;
            if ((lane & 7) == 0 && ch < cend) {
                const Val v = t.finish((uint64_t)keys[0]);
                if (c1 == 1)
                    v1 = v;
                else
                    mac(s2, keys[KEY_ROW + 1 + (ch - c0)], v);
            }
        }
        if (c1 == 1) {  // one chunk in all: its value is the hash
            if (lane == 0) store_result<N>(P, i, v1);
            continue;
        }
        s2 = warp_sum192(s2);
        Val w = {0, 0};
        if (lane == 0) {
            add192(s2, (uint64_t)keys[KEY_ROW], 0, 0);
            w = reduce<N>(s2);
        }
        if (levels == 2) {
            if (lane == 0) store_result<N>(P, i, w);
            continue;
        }
        // levels >= 3: the warp completing a node's children computes it
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
}

}  // namespace pm
