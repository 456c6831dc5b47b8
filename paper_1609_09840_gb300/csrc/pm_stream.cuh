// pm_stream.cuh -- one string hashed from pieces that arrive one after another.
//
// Sec. 4 notes that the tree of Algorithm 1 can be evaluated while the
// string is read once, keeping one incomplete chunk per level. Here the
// running state lives in device memory (StreamState) and every update is
// evaluated in parallel, level by level:
//   k_stream_l1    the complete level-1 chunks of an update (the chunk that
//                  the carried bytes start, completed by the piece's first
//                  bytes, then the chunks inside the piece, which may sit at
//                  any byte alignment), eight lanes per chunk: v = (b_1 + sum
//                  a_{1,i} s_i) mod p (Sec. 5, eq. 2wlinear; Sec. 6.2,
//                  Alg. 2); it also copies the piece's last incomplete chunk
//                  into the other carry buffer;
//   k_stream_fold  the level-1 values folded into level 2, one warp per
//                  chunk of level 2 that they touch: b_2 + sum a_{2,i} v_i of
//                  each completed chunk is reduced and becomes an input of
//                  level 3; the incomplete last chunk stays as a partial sum
//                  (double-buffered, so the warp that reads the old partial
//                  sum never races the one that writes the new one); the
//                  last block to finish does the same for levels 3 and up,
//                  a warp per touched chunk, one level after the other;
//                  k_stream_fold also folds, from level 3, the level-2
//                  values an update took straight from the tree kernel
//                  (pm_tree.cuh, level-2 output mode: the segment started a
//                  level-2 chunk); they wait in a buffer and are folded
//                  lazily (when it fills, before another update folds into
//                  level 3, and before a result);
//   k_stream_final the last chunk (carried bytes + the 0x01 pad of Sec. 4)
//                  and the completion of every level, exactly as the
//                  bounded-memory order of Sec. 4 finishes: the first level
//                  that received a single value holds the hash, partial
//                  chunks below it are zero-padded and hashed; then the
//                  output step (Sec. 5 end, Sec. 7). The state is not
//                  changed, so a string can be extended after a result.
// The host knows every count from the lengths alone (level L has received
// one value per completed chunk of level L - 1), so updates never wait for
// the device.
#pragma once
#include "pm_kernels.cuh"

namespace pm {

struct StreamState {
    U192 sum[2][LMAX + 2];     // partial sum of the incomplete chunk of each level (two buffers)
    uint32_t cnt[LMAX + 2];    // values in that chunk
    uint64_t total[LMAX + 2];  // values received by each level
    Val first[LMAX + 2];       // first value received by each level
    alignas(16) uint8_t carry[2][M * 8 + 16];  // bytes of the incomplete level-1 chunk (two buffers)
    unsigned arrive;                            // blocks of a level-2 fold that are done (0 between launches)
    unsigned long long tile_ctr;                // tiles claimed by the tree kernel's level-1 mode
};

// 8 bytes at any address p: the two aligned words around it, funnel-shifted
// (the bytes of those aligned words outside [p, p + 8) are read and ignored).
__device__ __forceinline__ uint64_t load8_any(const uint8_t *p) {
    const uintptr_t a = reinterpret_cast<uintptr_t>(p);
    const unsigned long long *q = reinterpret_cast<const unsigned long long *>(a & ~(uintptr_t)7);
    const uint32_t sh = (uint32_t)(a & 7) * 8;
    const uint64_t w0 = __ldg(q);
    if (sh == 0) return w0;
    const uint64_t w1 = __ldg(q + 1);
    return (w0 >> sh) | (w1 << (64 - sh));
}

// Unit u (bytes 8u .. 8u + 7) of the chunk made of the c carried bytes
// followed by the first bytes of the piece.
__device__ __forceinline__ uint64_t carried_unit(const uint8_t *carry, uint32_t c, const uint8_t *piece, uint32_t u) {
    const uint32_t o = 8 * u;
    if (o + 8 <= c) return *reinterpret_cast<const uint64_t *>(carry + o);
    if (o >= c) return load8_any(piece + (o - c));
    const uint32_t nlo = c - o;  // 1..7 carried bytes, then the piece's first bytes
    const uint64_t lo = *reinterpret_cast<const uint64_t *>(carry + o) & ((1ull << (8 * nlo)) - 1);
    return lo | (load8_any(piece) << (8 * nlo));
}

// Sum of an accumulator over each aligned group of G lanes, in the group's
// first lane (the other lanes keep partial sums).
template <int G>
__device__ __forceinline__ void group_sum(Acc32 &a) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) {
        a.L += __shfl_down_sync(0xffffffffu, a.L, d, G);
        a.H += __shfl_down_sync(0xffffffffu, a.H, d, G);
    }
}
template <int G>
__device__ __forceinline__ void group_sum(Acc64 &a) {
#pragma unroll
    for (int d = G / 2; d > 0; d >>= 1) {
        a.a00 += __shfl_down_sync(0xffffffffu, a.a00, d, G);
        a.a01 += __shfl_down_sync(0xffffffffu, a.a01, d, G);
        a.a10 += __shfl_down_sync(0xffffffffu, a.a10, d, G);
        a.a11 += __shfl_down_sync(0xffffffffu, a.a11, d, G);
        a.a20 += __shfl_down_sync(0xffffffffu, a.a20, d, G);
        a.a21 += __shfl_down_sync(0xffffffffu, a.a21, d, G);
    }
}

// Level-1 values of the chunks of one update segment: when carry_len > 0,
// chunk 0 is the carried bytes followed by the piece's first bytes; the
// others follow at `body` (any alignment). The segment that ends the update
// also copies the update's last `rem` bytes (at tail_src) into the other
// carry buffer, tail_dst. Eight lanes per chunk, four chunks per warp: lane j
// of a group takes units j, j + 8, j + 16, ... of its chunk (the group reads
// 64 contiguous bytes per load) with the split key words of those positions
// from shared memory; the group's partial sums meet in three shuffle steps
// and its first lane reduces (Sec. 6.2, Alg. 2) and stores.
constexpr int SL_GROUP = 8;  // lanes per chunk

template <int N>
__global__ void __launch_bounds__(256, N == 64 ? 4 : 5) k_stream_l1(const typename Fam<N>::word *gkey,
                                                                 const uint8_t *carry, uint32_t carry_len,
                                                                 const uint8_t *piece, const uint8_t *body,
                                                                 uint64_t nbody, const uint8_t *tail_src,
                                                                 uint32_t rem, uint8_t *tail_dst, Val *out) {
    typedef typename AccT<N>::t Acc;
    constexpr int UNITS = M * Fam<N>::W / 8;           // 8-byte units per chunk: 64 or 128
    constexpr int UPL = UNITS / SL_GROUP;              // units per lane: 8 or 16
    static_assert(UPL % 8 == 0, "units per lane in steps of eight");
    constexpr int CPW = 32 / SL_GROUP;                 // chunks per warp
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;  // chunk bytes
    __shared__ uint4 ks[UNITS];                        // split key words of unit u
    __shared__ uint64_t b1;
    for (int u = threadIdx.x; u < UNITS; u += blockDim.x) ks[u] = split_group<N>(gkey + 1, u);
    if (threadIdx.x == 0) b1 = (uint64_t)gkey[0];
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = gt; i < rem; i += (uint64_t)gridDim.x * blockDim.x) tail_dst[i] = tail_src[i];
    __syncthreads();
    const int lane = threadIdx.x & 31, grp = lane / SL_GROUP, j = lane % SL_GROUP;
    const int use_carry = carry_len ? 1 : 0;
    const uint64_t n = (uint64_t)use_carry + nbody;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    const bool aligned = (reinterpret_cast<uintptr_t>(body) & 7) == 0;  // every chunk of the piece alike
    for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w * CPW < n; w += nw) {
        const uint64_t c = w * CPW + grp;
        const bool have = c < n;
        const bool from_carry = use_carry && c == 0;
        const uint8_t *p = from_carry ? piece : body + (have ? c - (uint64_t)use_carry : 0) * CB;
        Acc acc;
        acc.zero();
        // eight units per lane at a time: their loads are issued together.
        // Whole 8-byte words when the piece is 8-byte aligned and the warp
        // has no carried chunk (the common case), else the general reads.
        if (aligned && !(use_carry && w == 0)) {
            const unsigned long long *q = reinterpret_cast<const unsigned long long *>(p);
#pragma unroll 1
            for (int t0 = 0; t0 < UPL; t0 += 8) {
                uint64_t x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) x[t] = have ? __ldg(q + j + SL_GROUP * (t0 + t)) : 0ull;
#pragma unroll
                for (int t = 0; t < 8; ++t) add_unit(acc, ks[j + SL_GROUP * (t0 + t)], x[t]);
            }
        } else {
#pragma unroll 1
            for (int t0 = 0; t0 < UPL; t0 += 8) {
                uint64_t x[8];
#pragma unroll
                for (int t = 0; t < 8; ++t) {
                    const uint32_t u = (uint32_t)(j + SL_GROUP * (t0 + t));
                    x[t] = !have ? 0ull : from_carry ? carried_unit(carry, carry_len, piece, u) : load8_any(p + 8 * u);
                }
#pragma unroll
                for (int t = 0; t < 8; ++t) add_unit(acc, ks[j + SL_GROUP * (t0 + t)], x[t]);
            }
        }
        group_sum<SL_GROUP>(acc);
        if (j == 0 && have) out[c] = acc.finish(b1);
    }
}

// Fold the n_in values of level L-1 (in[], the values number c_old ..
// c_old + n_in - 1 that level L receives) into level L, chunk k0 + w of
// level L by warp w of nw. Every completed chunk k of level L writes its value
// to out[k - c_old / m]; the partial sum of the incomplete chunk is read from
// sum[src][L] and written to sum[src ^ 1][L]. Returns the number of values
// written.
template <int N>
__device__ __forceinline__ uint64_t fold_level(StreamState *st, const typename Fam<N>::word *gkey, int L,
                                               const Val *in, uint64_t c_old, uint64_t n_in, int src, Val *out,
                                               uint64_t w0, uint64_t nw) {
    typedef typename Fam<N>::word word;
    const int lane = threadIdx.x & 31;
    const word *row = gkey + (size_t)(L - 1) * KEY_ROW;  // b_L, a_{L,1..m}
    const uint64_t c_new = c_old + n_in;
    const uint64_t k0 = c_old / M, k1 = (c_new - 1) / M;
    for (uint64_t w = w0; w <= k1 - k0; w += nw) {
        const uint64_t k = k0 + w;
        const uint64_t lo = k * M > c_old ? k * M : c_old;
        const uint64_t hi = (k + 1) * M < c_new ? (k + 1) * M : c_new;
        U192 s = {0, 0, 0};
        for (uint64_t pos = lo + lane; pos < hi; pos += 32) mac(s, row[1 + (pos - k * M)], in[pos - c_old]);
        s = warp_sum192(s);
        if (lane == 0) {
            if (k * M < c_old) add192(s, st->sum[src][L]);  // the chunk's earlier values
            if (hi == (k + 1) * M) {
                add192(s, (uint64_t)row[0], 0, 0);
                out[k - k0] = reduce<N>(s);
                if (k == k1) st->sum[src ^ 1][L] = U192{0, 0, 0};
            } else {
                st->sum[src ^ 1][L] = s;
            }
            if (k == k0) {
                if (c_old == 0) st->first[L] = in[0];
                st->total[L] = c_new;
                st->cnt[L] = (uint32_t)(c_new % M);
            }
        }
    }
    return c_new / M - k0;
}

// Levels 3 and up, one after the other, by the warps of one block (an update
// segment gives level 3 at most m^-1 of its level-1 values). c_old[L]: values
// level L held before; cur: bit L selects the partial sum buffer of level L;
// the values of each level go to a and b in turn.
struct FoldRest {
    uint64_t c_old[LMAX + 2];
    uint32_t cur;
};

template <int N>
__device__ __forceinline__ void fold_rest(StreamState *st, const typename Fam<N>::word *gkey, const Val *in,
                                          uint64_t n_in, const FoldRest &fr, Val *a, Val *b, int L0 = 3) {
    uint64_t n = n_in;
    const Val *src = in;
    for (int L = L0; n > 0 && L <= LMAX; ++L) {
        Val *dst = (L & 1) ? a : b;
        n = fold_level<N>(st, gkey, L, src, fr.c_old[L], n, (int)((fr.cur >> L) & 1), dst, threadIdx.x >> 5,
                          blockDim.x / 32);
        __syncthreads();  // level L's values are complete before level L + 1 reads them
        src = dst;
    }
}

// Level lv (2 for an update's level-1 values, 3 for level-2 values that
// waited), one warp per chunk of level lv that the new values touch (their n2
// completed values go to out); then, when n2 > 0, the last block to finish
// (an arrival counter, no waiting) folds levels lv + 1 and up, reading those
// values and writing its levels to a and out in turn.
template <int N>
__global__ void __launch_bounds__(256) k_stream_fold(StreamState *st, const typename Fam<N>::word *gkey, int lv,
                                                     const Val *in, uint64_t c_old, uint64_t n_in, int src,
                                                     Val *out, uint64_t n2, const FoldRest fr, Val *a) {
    fold_level<N>(st, gkey, lv, in, c_old, n_in, src, out,
                  (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), (uint64_t)gridDim.x * (blockDim.x / 32));
    if (n2 == 0) return;
    __shared__ bool last;
    __threadfence();  // this block's level-2 values and state before its arrival
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->arrive, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) st->arrive = 0;
    fold_rest<N>(st, gkey, out, n2, fr, lv & 1 ? out : a, lv & 1 ? a : out, lv + 1);
}

// Values received so far by each level (the host's counts).
struct StreamCounts {
    uint64_t total[LMAX + 2];
};

// The last level-1 chunk (the carried bytes, the pad, zeros), then the
// completion of the tree and the output step, by one warp. cur: bit L selects
// the partial sum buffer of level L; counts: values each level has received.
// keys: shared memory holding the key rows of all levels (see load_key_rows).
template <int N>
__device__ __forceinline__ void stream_final_warp(const StreamState *st, const typename Fam<N>::word *keys,
                                                  int cb, uint32_t carry_len, uint32_t cur,
                                                  const StreamCounts &counts, void *out, uint64_t *raw) {
    typedef typename AccT<N>::t Acc;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;
    const int lane = threadIdx.x & 31;
    Acc acc;
    acc.zero();
#pragma unroll
    for (int q = 0; q < UPL; ++q) {
        const int u = lane + 32 * q;
        add_unit(acc, split_group<N>(keys + 1, u), load_unit_padded(st->carry[cb], carry_len, (uint64_t)u));
    }
    warp_allsum(acc);
    if (lane != 0) return;
    const Val v = acc.finish((uint64_t)keys[0]);
    LevelStream<N> ls;
    for (int j = 0; j < LMAX + 2; ++j) {
        ls.sum[j] = st->sum[(cur >> j) & 1][j];
        ls.total[j] = counts.total[j];
        ls.cnt[j] = (uint32_t)(counts.total[j] % M);
        ls.first[j] = st->first[j];
    }
    ls.push(2, v, keys);
    write_output<N>(out, raw, 0, ls.finish(keys));
}

// The key rows of all levels into shared memory by the first `threads`
// threads, every load in flight at once.
template <int N, int T>
__device__ __forceinline__ void load_key_rows(const typename Fam<N>::word *gkey, typename Fam<N>::word *keys) {
    typedef typename Fam<N>::word word;
    constexpr int KPT = (LMAX * KEY_ROW + T - 1) / T;
    word kw[KPT];
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        const int i = (int)threadIdx.x + T * q;
        kw[q] = i < LMAX * KEY_ROW ? gkey[i] : 0;
    }
#pragma unroll
    for (int q = 0; q < KPT; ++q) {
        const int i = (int)threadIdx.x + T * q;
        if (i < LMAX * KEY_ROW) keys[i] = kw[q];
    }
}

template <int N>
__global__ void __launch_bounds__(32) k_stream_final(const StreamState *st, const typename Fam<N>::word *gkey,
                                                     int cb, uint32_t carry_len, uint32_t cur,
                                                     const StreamCounts counts, void *out, uint64_t *raw) {
    __shared__ typename Fam<N>::word keys[LMAX * KEY_ROW];
    load_key_rows<N, 32>(gkey, keys);
    __syncwarp();
    // launched as a programmatic dependent: the launch before it on the stream
    // is complete, its writes visible, past this point
    asm volatile("griddepcontrol.wait;" ::: "memory");
    stream_final_warp<N>(st, keys, cb, carry_len, cur, counts, out, raw);
}

// The result of a string whose level-2 values still wait (the level-2 mode of
// the tree kernel): the fold of those values into level 3 and up, as
// k_stream_fold with lv = 3, and then, in the last block to finish, the final
// chunk and the completion of the tree by its first warp (one launch instead
// of two). cur and counts: the state after the fold.
template <int N>
__global__ void __launch_bounds__(256) k_stream_finish(StreamState *st, const typename Fam<N>::word *gkey,
                                                       const Val *in, uint64_t c_old, uint64_t n_in, int src,
                                                       Val *out, uint64_t n2, const FoldRest fr, Val *a, int cb,
                                                       uint32_t carry_len, uint32_t cur,
                                                       const StreamCounts counts, void *res, uint64_t *raw) {
    __shared__ typename Fam<N>::word keys[LMAX * KEY_ROW];
    __shared__ bool last;
    load_key_rows<N, 256>(gkey, keys);  // for the final chunk, should this block finish last
    // launched as a programmatic dependent of the last update's tree launch:
    // its level-2 values and state are complete and visible past this point
    asm volatile("griddepcontrol.wait;" ::: "memory");
    fold_level<N>(st, gkey, 3, in, c_old, n_in, src, out,
                  (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), (uint64_t)gridDim.x * (blockDim.x / 32));
    __threadfence();  // this block's level-3 values and state before its arrival
    __syncthreads();
    if (threadIdx.x == 0) last = atomicAdd(&st->arrive, 1u) == gridDim.x - 1;
    __syncthreads();
    if (!last) return;
    __threadfence();
    if (threadIdx.x == 0) st->arrive = 0;
    fold_rest<N>(st, gkey, out, n2, fr, out, a, 4);  // level 4 into a, level 5 into out, ...
    __syncthreads();
    __threadfence_block();
    if (threadIdx.x < 32) stream_final_warp<N>(st, keys, cb, carry_len, cur, counts, res, raw);
}

}  // namespace pm
