// pm_stream.cuh -- one string hashed from pieces that arrive one after another.
//
// Sec. 4 notes that the tree of Algorithm 1 can be evaluated while the
// string is read once, keeping one incomplete chunk per level. Here the
// running state lives in device memory (StreamState) and every update is
// evaluated in parallel, level by level:
//   k_stream_l1    the complete level-1 chunks of an update (the chunk that
//                  the carried bytes start, then the chunks inside the
//                  piece, which may sit at any byte alignment), one warp per
//                  chunk: v = (b_1 + sum a_{1,i} s_i) mod p (Sec. 5, eq.
//                  2wlinear; Sec. 6.2, Alg. 2);
//   k_stream_fold  the values of level L-1 folded into level L, one warp per
//                  chunk of level L that they touch: b_L + sum a_{L,i} v_i of
//                  each completed chunk is reduced and becomes an input of
//                  level L + 1; the incomplete last chunk stays as a partial
//                  sum (double-buffered, so the warp that reads the old
//                  partial sum never races the one that writes the new one);
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
    alignas(16) uint8_t carry[M * 8 + 16];  // bytes of the incomplete level-1 chunk
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

// Level-1 values of the chunks of one update: chunk 0 is the carry buffer
// when use_carry is set, the others follow at `body` (any alignment).
template <int N>
__global__ void __launch_bounds__(256) k_stream_l1(const typename Fam<N>::word *gkey, const uint8_t *carry,
                                                   int use_carry, const uint8_t *body, uint64_t nbody,
                                                   Val *out) {
    typedef typename AccT<N>::t Acc;
    typedef typename Fam<N>::word word;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;     // 8-byte units per lane per chunk: 2 or 4
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;  // chunk bytes
    __shared__ word keys[KEY_ROW];
    for (int i = threadIdx.x; i < KEY_ROW; i += blockDim.x) keys[i] = gkey[i];
    __syncthreads();
    const int lane = threadIdx.x & 31;
    uint4 kr[UPL];
#pragma unroll
    for (int q = 0; q < UPL; ++q) kr[q] = split_group<N>(keys + 1, lane + 32 * q);
    const uint64_t n = (uint64_t)use_carry + nbody;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t c = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); c < n; c += nw) {
        const bool from_carry = use_carry && c == 0;
        const uint8_t *p = from_carry ? carry : body + (c - (uint64_t)use_carry) * CB;
        uint64_t x[UPL];
#pragma unroll
        for (int q = 0; q < UPL; ++q) {
            const uint8_t *u = p + 8 * (lane + 32 * q);
            x[q] = from_carry ? *reinterpret_cast<const uint64_t *>(u) : load8_any(u);
        }
        Acc acc;
        acc.zero();
#pragma unroll
        for (int q = 0; q < UPL; ++q) add_unit(acc, kr[q], x[q]);
        warp_allsum(acc);
        if (lane == 0) out[c] = acc.finish((uint64_t)keys[0]);
    }
}

// Fold n_in values of level L-1 (in[], the values number c_old .. c_old +
// n_in - 1 that level L receives) into level L. Every completed chunk k of
// level L writes its value to out[k - c_old / m]; the partial sum of the
// incomplete chunk is read from sum[src][L] and written to sum[src ^ 1][L].
template <int N>
__global__ void __launch_bounds__(256) k_stream_fold(StreamState *st, const typename Fam<N>::word *gkey, int L,
                                                     const Val *in, uint64_t c_old, uint64_t n_in, int src,
                                                     Val *out) {
    typedef typename Fam<N>::word word;
    const int lane = threadIdx.x & 31;
    const word *row = gkey + (size_t)(L - 1) * KEY_ROW;  // b_L, a_{L,1..m}
    const uint64_t c_new = c_old + n_in;
    const uint64_t k0 = c_old / M, k1 = (c_new - 1) / M;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    for (uint64_t w = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); w <= k1 - k0; w += nw) {
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
}

// The last level-1 chunk (the carried bytes, the pad, zeros), then the
// completion of the tree and the output step. cur: bit L selects the partial
// sum buffer of level L. One warp.
template <int N>
__global__ void __launch_bounds__(32) k_stream_final(const StreamState *st, const typename Fam<N>::word *gkey,
                                                     uint32_t carry_len, uint32_t cur, void *out, uint64_t *raw) {
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
        add_unit(acc, split_group<N>(keys + 1, u), load_unit_padded(st->carry, carry_len, (uint64_t)u));
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
