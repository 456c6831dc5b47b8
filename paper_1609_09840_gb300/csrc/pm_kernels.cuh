// pm_kernels.cuh -- the CUDA kernels of PM+ hashing (arXiv 1609.09840).
//
//   k_keygen      key expansion (one thread, setup only)
//   (the single-buffer tree kernel k_tree is in pm_tree.cuh)
//   (the batched kernels are in pm_lane.cuh and pm_long.cuh)
//   k_plain       one string per launch (comparison baseline): one warp hashes
//                 the whole string, tree levels combined on the fly in the
//                 bounded-memory order of Sec. 4 (running multiply-accumulate
//                 per level)
//   k_debug_reduce the reduction of Sec. 6.2 + Algorithm 2 on given sums
#pragma once
#include <cuda.h>

#include "pm_async.cuh"
#include "pm_device.cuh"

namespace pm {

// ---------------------------------------------------------------------------
// Key expansion. Level-major rows (b_j, a_{j,1..m}); splitmix64 stream from
// `seed`; b = top n bits of a draw; a_i redrawn until in [1, p - kappa - 1].
// ---------------------------------------------------------------------------
template <int N>
__global__ void k_keygen(uint64_t seed, typename Fam<N>::word *key) {
    typedef typename Fam<N>::word word;
    if (threadIdx.x != 0 || blockIdx.x != 0) return;
    const uint64_t wmax = N == 64 ? ~0ull : ((1ull << N) - 1);
    const uint64_t amax = wmax - (Fam<N>::KAPPA - Fam<N>::K);  // p - kappa - 1
    uint64_t draw = 0;
    for (int j = 0; j < LMAX; ++j) {
        key[j * KEY_ROW] = (word)(splitmix64_at(seed, draw++) >> (64 - N));
        for (int i = 1; i <= M; ++i) {
            uint64_t a;
            do {
                a = splitmix64_at(seed, draw++) >> (64 - N);
            } while (a < 1 || a > amax);
            key[j * KEY_ROW + i] = (word)a;
        }
    }
}

// ---------------------------------------------------------------------------
// Word i (0-based) of the padded string sigma of a byte string of `len` bytes
// at `p` (8-byte aligned), read as 8-byte units: unit u holds bytes
// [8u, 8u + 8). Sec. 4: the string is followed by a 0x01 byte and zeros.
// Only bytes of 8-byte words that contain string bytes are read.
// ---------------------------------------------------------------------------
__device__ __forceinline__ uint64_t load_unit_padded(const uint8_t *p, uint64_t len, uint64_t u) {
    const uint64_t off = u * 8;
    if (off + 8 <= len) return __ldg(reinterpret_cast<const unsigned long long *>(p + off));
    if (off > len) return 0;
    const uint32_t rem = (uint32_t)(len - off);  // 0..7 string bytes in this unit
    uint64_t x = 0;
    if (rem) x = __ldg(reinterpret_cast<const unsigned long long *>(p + off)) &
                 ((1ull << (8 * rem)) - 1);
    return x | (1ull << (8 * rem));
}

template <int N> struct KSplit;
template <> struct KSplit<32> { typedef uint4 t; static constexpr int COUNT = M / 2; };  // 2 words per uint4
template <> struct KSplit<64> { typedef uint4 t; static constexpr int COUNT = M; };      // 1 word per uint4
template <int N> struct AccT;
template <> struct AccT<32> { typedef Acc32 t; };
template <> struct AccT<64> { typedef Acc64 t; };

template <int N> struct AccCT;
template <> struct AccCT<32> { typedef AccC32 t; };
template <> struct AccCT<64> { typedef AccC64 t; };

// Key words of one 8-byte unit: two 32-bit words (n = 32) or one 64-bit word.
template <int N> struct UnitKey;
template <> struct UnitKey<32> { typedef uint2 t; };
template <> struct UnitKey<64> { typedef uint64_t t; };

// The key words of unit u of a level-1 chunk, from the key row b_1, a_{1,1..m}.
template <int N>
__device__ __forceinline__ typename UnitKey<N>::t unit_key(const typename Fam<N>::word *row, int u) {
    if constexpr (N == 32)
        return make_uint2((uint32_t)row[1 + 2 * u], (uint32_t)row[2 + 2 * u]);
    else
        return (uint64_t)row[1 + u];
}

// acc += a * x for the one or two words of the 8-byte unit x (carry chains).
__device__ __forceinline__ void add_unit_c(AccC32 &acc, const uint2 &k, uint64_t x) {
    acc.add(k.x, (uint32_t)x);
    acc.add(k.y, (uint32_t)(x >> 32));
}
__device__ __forceinline__ void add_unit_c(AccC64 &acc, uint64_t k, uint64_t x) { acc.add(k, x); }

// acc += products of the words of one 16-byte group d with the key words k
// of the same positions (4 words for n = 32, 2 for n = 64; little-endian).
__device__ __forceinline__ void add16c(AccC32 &acc, const uint4 &k, const uint4 &d) {
    acc.add(k.x, d.x);
    acc.add(k.y, d.y);
    acc.add(k.z, d.z);
    acc.add(k.w, d.w);
}
__device__ __forceinline__ void add16c(AccC64 &acc, const uint4 &k, const uint4 &d) {
    acc.add(((uint64_t)k.y << 32) | k.x, ((uint64_t)d.y << 32) | d.x);
    acc.add(((uint64_t)k.w << 32) | k.z, ((uint64_t)d.w << 32) | d.z);
}

// acc += products of one 16-byte group of words starting at word index w0.
__device__ __forceinline__ void add16(Acc32 &acc, const uint4 *keys1, int w0, const uint4 &d) {
    const uint4 ka = keys1[w0 / 2], kb = keys1[w0 / 2 + 1];  // (aL, aH) of 4 words
    acc.add(make_uint2(ka.x, ka.y), d.x);
    acc.add(make_uint2(ka.z, ka.w), d.y);
    acc.add(make_uint2(kb.x, kb.y), d.z);
    acc.add(make_uint2(kb.z, kb.w), d.w);
}
__device__ __forceinline__ void add16(Acc64 &acc, const uint4 *keys1, int w0, const uint4 &d) {
    acc.add(keys1[w0], (uint64_t)d.x | ((uint64_t)d.y << 32));
    acc.add(keys1[w0 + 1], (uint64_t)d.z | ((uint64_t)d.w << 32));
}
// acc += products of one 8-byte unit x given the split keys k of its words.
__device__ __forceinline__ void add_unit(Acc32 &acc, const uint4 &k, uint64_t x) {
    acc.add(make_uint2(k.x, k.y), (uint32_t)x);
    acc.add(make_uint2(k.z, k.w), (uint32_t)(x >> 32));
}
__device__ __forceinline__ void add_unit(Acc64 &acc, const uint4 &k, uint64_t x) { acc.add(k, x); }
// split key group g: for n = 32 the words 2g, 2g+1; for n = 64 the word g.
template <int N>
__device__ __forceinline__ uint4 split_group(const typename Fam<N>::word *a, int g) {
    if constexpr (N == 32) {
        const uint2 k0 = split_key32((uint32_t)a[2 * g]);
        const uint2 k1 = split_key32((uint32_t)a[2 * g + 1]);
        return make_uint4(k0.x, k0.y, k1.x, k1.y);
    } else {
        return split_key64((uint64_t)a[g]);
    }
}
// butterfly sum over the warp: every lane ends with the total
__device__ __forceinline__ void warp_allsum(Acc32 &a) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a.L += __shfl_xor_sync(0xffffffffu, a.L, d);
        a.H += __shfl_xor_sync(0xffffffffu, a.H, d);
    }
}
__device__ __forceinline__ void warp_allsum(Acc64 &a) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) {
        a.a00 += __shfl_xor_sync(0xffffffffu, a.a00, d);
        a.a01 += __shfl_xor_sync(0xffffffffu, a.a01, d);
        a.a10 += __shfl_xor_sync(0xffffffffu, a.a10, d);
        a.a11 += __shfl_xor_sync(0xffffffffu, a.a11, d);
        a.a20 += __shfl_xor_sync(0xffffffffu, a.a20, d);
        a.a21 += __shfl_xor_sync(0xffffffffu, a.a21, d);
    }
}

template <int N>
__device__ __forceinline__ void write_output(void *out, uint64_t *raw, uint64_t idx, const Val &h) {
    if constexpr (N == 32)
        static_cast<uint32_t *>(out)[idx] = mix32((uint32_t)h.lo);  // h mod 2^32, mixed
    else
        static_cast<uint64_t *>(out)[idx] = mix64(h.lo);            // h mod 2^64, mixed
    if (raw) {
        raw[2 * idx] = h.lo;
        raw[2 * idx + 1] = h.hi;
    }
}

// ---------------------------------------------------------------------------
// Ragged batch.
// ---------------------------------------------------------------------------
__device__ __forceinline__ void string_span(const int64_t *off, int64_t i, uint64_t &start,
                                            uint64_t &len) {
    const int64_t s = (__ldg(off + i) + 7) & ~(int64_t)7;
    const int64_t e = __ldg(off + i + 1);
    start = (uint64_t)s;
    len = e > s ? (uint64_t)(e - s) : 0;
}

__device__ __forceinline__ unsigned lanemask_lt() { return (1u << (threadIdx.x & 31)) - 1; }

// Units of a string that the batch tile kernel's first pass may take (its
// key words travel as launch parameters).
constexpr int BL_P1_MAX = 8;

struct BatchParams {
    uint4 k1[BL_P1_MAX];             // split level-1 key words of units 0..BL_P1_MAX-1
    uint64_t b1;                     // b_1
    const uint8_t *base;
    const int64_t *off;
    int64_t n;
    const void *key;
    void *out;                       // hashes (mode 0) or raw pairs (mode 1)
    unsigned *tile_ctr;              // tiles claimed by the tile kernel beyond the first per warp
    int raw;
    // work items of the strings of at least BIG_CHUNKS chunks (see pm_long.cuh)
    unsigned long long *big_count;   // segments reserved
    unsigned long long *big_next;    // segments claimed
    unsigned long long *pool_next;   // tree storage reserved (bytes)
    int64_t *big_str;                // string of each segment (-1: refused)
    int64_t *big_pool;               // tree storage of the string (byte offset), -1 if none
    int32_t *big_seg;                // segment number within the string
    uint8_t *pool;                   // tree storage
    uint64_t big_cap, pool_cap;      // capacities (a reservation beyond them is refused)
    int *status;                     // per-call device status word (may be null)
};

template <int N>
__device__ __forceinline__ void store_result(const BatchParams &P, int64_t i, const Val &h) {
    if (P.raw) {
        static_cast<uint64_t *>(P.out)[2 * i] = h.lo;
        static_cast<uint64_t *>(P.out)[2 * i + 1] = h.hi;
    } else {
        write_output<N>(P.out, nullptr, (uint64_t)i, h);
    }
}

// Running state of the tree levels >= 2 of one string: each level keeps the
// sum b_j + sum a_{j,i} v_i of its current chunk, so that the tree of
// Algorithm 1 is evaluated in the bounded-memory order of Sec. 4 with one
// accumulator per level instead of m stored values.
template <int N>
struct LevelStream {
    typedef typename Fam<N>::word word;
    U192 sum[LMAX + 2];
    uint32_t cnt[LMAX + 2];
    uint64_t total[LMAX + 2];
    Val first[LMAX + 2];

    __device__ __forceinline__ void init() {
#pragma unroll
        for (int j = 0; j < LMAX + 2; ++j) {
            sum[j] = U192{0, 0, 0};
            cnt[j] = 0;
            total[j] = 0;
            first[j] = Val{0, 0};
        }
    }
    // push the value v into level j (the input string of f_j)
    __device__ __forceinline__ void push(int j, Val v, const word *keys) {
        while (j <= LMAX) {
            if (total[j] == 0) first[j] = v;
            mac(sum[j], keys[(j - 1) * KEY_ROW + 1 + cnt[j]], v);
            ++cnt[j];
            ++total[j];
            if (cnt[j] < (uint32_t)M) return;
            U192 s = sum[j];
            add192(s, (uint64_t)keys[(j - 1) * KEY_ROW], 0, 0);
            v = reduce<N>(s);
            sum[j] = U192{0, 0, 0};
            cnt[j] = 0;
            ++j;
        }
        if (total[LMAX + 1] == 0) first[LMAX + 1] = v;
        ++total[LMAX + 1];
    }
    // Completion: the first level that received a single value holds the
    // hash; partial chunks below it are zero-padded and hashed.
    __device__ __forceinline__ Val finish(const word *keys) {
        for (int j = 2; j <= LMAX; ++j) {
            if (total[j] == 1) return first[j];
            if (cnt[j] > 0) {
                U192 s = sum[j];
                add192(s, (uint64_t)keys[(j - 1) * KEY_ROW], 0, 0);
                sum[j] = U192{0, 0, 0};
                cnt[j] = 0;
                push(j + 1, reduce<N>(s), keys);
            }
        }
        return first[LMAX + 1];
    }
};

// One warp hashes one whole string of any length. Lane l covers the 8-byte
// units l, l+32, l+64, l+96 of each 128-word chunk (PM+32 chunks have 64
// units); level-1 key words stay in registers.
template <int N>
__device__ __forceinline__ Val warp_hash_string(const uint8_t *p, uint64_t len,
                                                const typename Fam<N>::word *keys) {
    typedef typename AccT<N>::t Acc;
    const int lane = threadIdx.x & 31;
    constexpr int UPL = (M * Fam<N>::W / 8) / 32;  // units per lane per chunk: 2 or 4
    uint4 kr[UPL];
#pragma unroll
    for (int q = 0; q < UPL; ++q) kr[q] = split_group<N>(keys + 1, lane + 32 * q);
    const uint64_t n0 = len / Fam<N>::W + 1;
    const uint64_t nchunks = (n0 + M - 1) / M;
    const uint64_t chunk_bytes = (uint64_t)M * Fam<N>::W;
    // Strings of at most m level-1 chunks (two levels): the level-2 sum
    // b_2 + sum a_{2,c} v_c is kept in registers. Longer strings feed the
    // running per-level sums of LevelStream.
    const bool two_levels = nchunks <= (uint64_t)M;
    LevelStream<N> st;
    if (!two_levels) st.init();
    U192 s2 = {0, 0, 0};
    Val v1 = {0, 0};
    // the loads of chunk c+1 are issued before chunk c is reduced
    uint64_t xn[UPL];
#pragma unroll
    for (int q = 0; q < UPL; ++q) xn[q] = load_unit_padded(p, len, (uint64_t)(lane + 32 * q));
    for (uint64_t c = 0; c < nchunks; ++c) {
        uint64_t x[UPL];
#pragma unroll
        for (int q = 0; q < UPL; ++q) x[q] = xn[q];
        if (c + 1 < nchunks) {
            const uint8_t *cp = p + (c + 1) * chunk_bytes;
            const uint64_t clen = len - (c + 1) * chunk_bytes;  // bytes from that chunk on
#pragma unroll
            for (int q = 0; q < UPL; ++q) xn[q] = load_unit_padded(cp, clen, (uint64_t)(lane + 32 * q));
        }
        Acc acc;
        acc.zero();
#pragma unroll
        for (int q = 0; q < UPL; ++q) add_unit(acc, kr[q], x[q]);
        warp_allsum(acc);
        const Val v = acc.finish((uint64_t)keys[0]);
        if (nchunks == 1)
            v1 = v;
        else if (two_levels)
            mac(s2, keys[KEY_ROW + 1 + c], v);
        else
            st.push(2, v, keys);
    }
    if (nchunks == 1) return v1;
    if (two_levels) {
        add192(s2, (uint64_t)keys[KEY_ROW], 0, 0);
        return reduce<N>(s2);
    }
    return st.finish(keys);
}

// One launch per string (the plain comparison path): one warp.
template <int N>
__global__ void __launch_bounds__(32) k_plain(const uint8_t *base, const int64_t *off, int64_t i,
                                              const typename Fam<N>::word *gkey, void *out) {
    typedef typename Fam<N>::word word;
    __shared__ word keys[LMAX * KEY_ROW];
    for (int t = threadIdx.x; t < LMAX * KEY_ROW; t += 32) keys[t] = gkey[t];
    __syncwarp();
    uint64_t start, len;
    string_span(off, i, start, len);
    const Val h = warp_hash_string<N>(base + start, len, keys);
    if (threadIdx.x == 0) write_output<N>(out, nullptr, (uint64_t)i, h);
}

template <int N>
__global__ void k_debug_reduce(const uint64_t *S, int64_t n, uint64_t *z) {
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    U192 s = {S[3 * i], S[3 * i + 1], S[3 * i + 2]};
    const Val v = reduce<N>(s);
    z[2 * i] = v.lo;
    z[2 * i + 1] = v.hi;
}

}  // namespace pm
