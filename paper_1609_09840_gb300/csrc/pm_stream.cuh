// pm_stream.cuh -- one string hashed from pieces that arrive one after another.
//
// Sec. 4 notes that the tree of Algorithm 1 can be evaluated while the
// string is read once, keeping one incomplete chunk per level. Here the
// running state lives in device memory (StreamState) and every update is
// evaluated in parallel, level by level:
//   k_stream_l1    the complete level-1 chunks of an update (the chunk that
//                  the carried bytes start, completed by the piece's first
//                  bytes, then the chunks inside the piece, which may sit at
//                  any byte alignment), one warp per chunk: v = (b_1 + sum
//                  a_{1,i} s_i) mod p (Sec. 5, eq. 2wlinear; Sec. 6.2,
//                  Alg. 2); it also copies the piece's last incomplete chunk
//                  into the other carry buffer;
//   k_stream_fold  the level-1 values folded into level 2, one warp per
//                  chunk of level 2 that they touch: b_2 + sum a_{2,i} v_i of
//                  each completed chunk is reduced and becomes an input of
//                  level 3; the incomplete last chunk stays as a partial sum
//                  (double-buffered, so the warp that reads the old partial
//                  sum never races the one that writes the new one);
//   k_stream_fold_rest  the same for levels 3 and up, by one warp;
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

// Level-1 values of the chunks of one update segment: when carry_len > 0,
// chunk 0 is the carried bytes followed by the piece's first bytes; the
// others follow at `body` (any alignment). The segment that ends the update
// also copies the update's last `rem` bytes (at tail_src) into the other
// carry buffer, tail_dst.
template <int N>
__global__ void __launch_bounds__(256) k_stream_l1(const typename Fam<N>::word *gkey, const uint8_t *carry,
                                                   uint32_t carry_len, const uint8_t *piece, const uint8_t *body,
                                                   uint64_t nbody, const uint8_t *tail_src, uint32_t rem,
                                                   uint8_t *tail_dst, Val *out) {
    typedef typename AccT<N>::t Acc;
    typedef typename Fam<N>::word word;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;     // 8-byte units per lane per chunk: 2 or 4
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;  // chunk bytes
    __shared__ word keys[KEY_ROW];
    for (int i = threadIdx.x; i < KEY_ROW; i += blockDim.x) keys[i] = gkey[i];
    const uint64_t gt = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (uint64_t i = gt; i < rem; i += (uint64_t)gridDim.x * blockDim.x) tail_dst[i] = tail_src[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint4 kr[UPL];
#pragma unroll
    for (int q = 0; q < UPL; ++q) kr[q] = split_group<N>(keys + 1, lane + 32 * q);
    const int use_carry = carry_len ? 1 : 0;
    const uint64_t n = (uint64_t)use_carry + nbody;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); c < n; c += nw) {
        const bool from_carry = use_carry && c == 0;
        const uint8_t *p = from_carry ? piece : body + (c - (uint64_t)use_carry) * CB;
        uint64_t x[UPL];
#pragma unroll
        for (int q = 0; q < UPL; ++q) {
            const uint32_t u = (uint32_t)(lane + 32 * q);
            x[q] = from_carry ? carried_unit(carry, carry_len, piece, u) : load8_any(p + 8 * u);
        }
        Acc acc;
        acc.zero();
#pragma unroll
        for (int q = 0; q < UPL; ++q) add_unit(acc, kr[q], x[q]);
        warp_allsum(acc);
        if (lane == 0) out[c] = acc.finish((uint64_t)keys[0]);
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

// Level 2: one warp per chunk of level 2 that the new level-1 values touch.
template <int N>
__global__ void __launch_bounds__(256) k_stream_fold(StreamState *st, const typename Fam<N>::word *gkey,
                                                     const Val *in, uint64_t c_old, uint64_t n_in, int src,
                                                     Val *out) {
    fold_level<N>(st, gkey, 2, in, c_old, n_in, src, out,
                  (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5), (uint64_t)gridDim.x * (blockDim.x / 32));
}

// Levels 3 and up, one after the other, by one warp (an update segment
// gives level 3 at most m^-1 of its level-1 values). c_old[L]: values level
// L held before; cur: bit L selects the partial sum buffer of level L; the
// values of each level go to a and b in turn.
struct FoldRest {
    uint64_t c_old[LMAX + 2];
    uint32_t cur;
};

template <int N>
__global__ void __launch_bounds__(32) k_stream_fold_rest(StreamState *st, const typename Fam<N>::word *gkey,
                                                         const Val *in, uint64_t n_in, const FoldRest fr, Val *a,
                                                         Val *b) {
    uint64_t n = n_in;
    const Val *src = in;
    for (int L = 3; n > 0 && L <= LMAX; ++L) {
        Val *dst = (L & 1) ? a : b;
        n = fold_level<N>(st, gkey, L, src, fr.c_old[L], n, (int)((fr.cur >> L) & 1), dst, 0, 1);
        __syncwarp();
        src = dst;
    }
}

// The last level-1 chunk (the carried bytes, the pad, zeros), then the
// completion of the tree and the output step. cur: bit L selects the partial
// sum buffer of level L. One warp.
template <int N>
__global__ void __launch_bounds__(32) k_stream_final(const StreamState *st, const typename Fam<N>::word *gkey,
                                                     int cb, uint32_t carry_len, uint32_t cur, void *out,
                                                     uint64_t *raw) {
    typedef typename AccT<N>::t Acc;
    typedef typename Fam<N>::word word;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;
    __shared__ word keys[LMAX * KEY_ROW];
    for (int i = threadIdx.x; i < LMAX * KEY_ROW; i += 32) keys[i] = gkey[i];
    __syncwarp();
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
        ls.cnt[j] = st->cnt[j];
        ls.total[j] = st->total[j];
        ls.first[j] = st->first[j];
    }
    ls.push(2, v, keys);
    write_output<N>(out, raw, 0, ls.finish(keys));
}

}  // namespace pm
