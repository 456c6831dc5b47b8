// pm_toy.cuh -- toy members of the PM+ family, evaluated exhaustively on the
// device to check the family's two properties at sizes where every case can
// be enumerated.
//
// Sec. 5 defines PM+-Multilinear for any prime p with 2^n the largest power
// of two below it; its table of the smallest primes above powers of two
// starts with 2^8 + 1 and 2^16 + 1 (k = 1). With n = 8 or 16 the words are
// one or two bytes, so a word position can take every one of its 2^n values
// and a one-chunk function can take every key:
//   k_toy_regular  component-wise regularity (Sec. 3 definitions; Sec. 5:
//                  with every a_i non-zero, f(s) = y has exactly one solution
//                  in each component): for one key and one word position of a
//                  byte string, all 2^n values of that word are hashed by
//                  the whole tree of Algorithm 1 (padding of Sec. 4); the raw
//                  values must be pairwise distinct, and after mod 2^n (Sec. 3,
//                  the lemma on reducing mod M) no value may have more than two
//                  preimages and at most k values two;
//   k_toy_delta    almost Delta-universality (Sec. 5): for two inputs s != t
//                  of a one-chunk function, every key (a_1 .. a_m) in
//                  [1, p - kappa - 1]^m, the histogram of f(s) - f(t) mod p; no
//                  difference may occur for more than a 1 / (p - 1 - kappa)
//                  fraction of the keys.
// The values are below 2^17, so every chunk sum is formed exactly in 64 bits
// and reduced by the integer remainder: at these sizes the definition itself
// (eq. 2wlinear) is the cheapest form. Keys follow the library convention
// (splitmix64 of the seed; per level b_j = the top n bits of a draw, then
// a_{j,i} = the top n bits of the next draws, redrawn until in [1, p - kappa - 1]).
#pragma once
#include "pm_device.cuh"

namespace pm {

constexpr int TOY_MAXM = 16;      // chunk length m
constexpr int TOY_MAXL = 8;       // levels L
constexpr int TOY_MAXW = 128;     // level-1 words of a string (with the pad word)
constexpr int TOY_THREADS = 256;

struct ToyParams {
    uint32_t n, k, kappa, m, L;
};

__device__ __forceinline__ uint32_t toy_prime(const ToyParams &P) { return (1u << P.n) + P.k; }

// Largest key word the convention draws: p - kappa - 1 when that is an n-bit
// value, else 2^n - 1 (every non-zero n-bit value).
__host__ __device__ __forceinline__ uint32_t toy_amax(const ToyParams &P) {
    const uint32_t wmax = (1u << P.n) - 1;
    return P.kappa >= P.k ? wmax - (P.kappa - P.k) : wmax;
}

// Level-major key: level j at key[j (1 + m)] = b_j, a_{j,1} .. a_{j,m}.
__device__ void toy_key(const ToyParams &P, uint64_t seed, uint32_t *key) {
    const uint32_t amax = toy_amax(P);
    uint64_t draw = 0;
    for (uint32_t j = 0; j < P.L; ++j) {
        uint32_t *f = key + j * (1 + P.m);
        f[0] = (uint32_t)(splitmix64_at(seed, draw++) >> (64 - P.n));
        for (uint32_t i = 1; i <= P.m; ++i) {
            uint32_t a;
            do {
                a = (uint32_t)(splitmix64_at(seed, draw++) >> (64 - P.n));
            } while (a < 1 || a > amax);
            f[i] = a;
        }
    }
}

// Algorithm 1 on the word string v[0 .. N) (the pad word included), in
// place: each level replaces the string by the values of its m-word chunks
// (the last one zero-padded), f_j(s) = (b_j + sum a_{j,i} s_i) mod p, at
// least once, until one value is left.
__device__ uint32_t toy_tree(const ToyParams &P, const uint32_t *key, uint32_t *v, uint32_t N) {
    const uint64_t p = toy_prime(P);
    uint32_t j = 0;
    do {
        const uint32_t *f = key + j * (1 + P.m);
        const uint32_t nc = (N + P.m - 1) / P.m;
        for (uint32_t c = 0; c < nc; ++c) {
            uint64_t s = f[0];
            for (uint32_t i = 0; i < P.m && c * P.m + i < N; ++i) s += (uint64_t)f[1 + i] * v[c * P.m + i];
            v[c] = (uint32_t)(s % p);
        }
        N = nc;
        ++j;
    } while (N > 1);
    return v[0];
}

// One block per (key, word position): key q is the key of seed seed0 + q,
// position c = comp0 + the block's position index. str: len bytes, the
// string whose word c takes every value x in [0, 2^n). Per block, counts[3]
// = {raw values already seen, values mod 2^n seen a second time, values mod
// 2^n seen a third time or more}; raw (optional) receives the 2^n raw values.
__global__ void __launch_bounds__(TOY_THREADS) k_toy_regular(ToyParams P, uint64_t seed0, uint32_t ncomp,
                                                             uint32_t comp0, const uint8_t *str, uint32_t len,
                                                             uint32_t *counts, uint32_t *raw) {
    __shared__ uint32_t key[TOY_MAXL * (1 + TOY_MAXM)];
    __shared__ uint32_t words[TOY_MAXW];
    __shared__ uint32_t seen_raw[((1u << 16) + 1 + 31) / 32], seen1[(1u << 16) / 32], seen2[(1u << 16) / 32];
    __shared__ uint32_t cnt[3];
    const uint32_t q = blockIdx.x / ncomp, c = comp0 + blockIdx.x % ncomp;
    const uint32_t W = P.n / 8, N0 = len / W + 1, X = 1u << P.n, p = toy_prime(P);
    if (threadIdx.x == 0) toy_key(P, seed0 + q, key);
    // the padded words (Sec. 4): little-endian bytes, then 0x01, then zeros
    for (uint32_t i = threadIdx.x; i < N0; i += blockDim.x) {
        uint32_t w = 0;
        for (uint32_t b = 0; b < W; ++b) {
            const uint32_t pos = i * W + b;
            const uint32_t byte = pos < len ? str[pos] : (pos == len ? 1u : 0u);
            w |= byte << (8 * b);
        }
        words[i] = w;
    }
    for (uint32_t i = threadIdx.x; i < (p + 31) / 32; i += blockDim.x) seen_raw[i] = 0;
    for (uint32_t i = threadIdx.x; i < X / 32; i += blockDim.x) seen1[i] = seen2[i] = 0;
    if (threadIdx.x < 3) cnt[threadIdx.x] = 0;
    __syncthreads();
    uint32_t v[TOY_MAXW];
    for (uint32_t x = threadIdx.x; x < X; x += blockDim.x) {
        for (uint32_t i = 0; i < N0; ++i) v[i] = words[i];
        v[c] = x;
        const uint32_t h = toy_tree(P, key, v, N0);
        if (raw) raw[(size_t)blockIdx.x * X + x] = h;
        if (atomicOr(&seen_raw[h >> 5], 1u << (h & 31)) & (1u << (h & 31))) atomicAdd(&cnt[0], 1u);
        const uint32_t z = h & (X - 1), bit = 1u << (z & 31);
        if (atomicOr(&seen1[z >> 5], bit) & bit) {
            if (atomicOr(&seen2[z >> 5], bit) & bit)
                atomicAdd(&cnt[2], 1u);
            else
                atomicAdd(&cnt[1], 1u);
        }
    }
    __syncthreads();
    if (threadIdx.x < 3) counts[(size_t)blockIdx.x * 3 + threadIdx.x] = cnt[threadIdx.x];
}

// The differences d_i = (s_i - t_i) mod p of the two inputs, component 0
// first among those with d_i != 0 (the component the lanes step through).
struct ToyDelta {
    uint32_t d[TOY_MAXM];
};

// hist[e] += the number of keys (a_1 .. a_m) in [1, R]^m, R = p - kappa - 1,
// with sum a_i d_i = e (mod p), i.e. f(s) - f(t) = e (b cancels). One warp per
// value of (a_2 .. a_m) (mixed radix R, index o < R^(m-1)); its lanes step a_1
// through [1, R] by 32, the difference advancing by 32 d_1 mod p.
__global__ void __launch_bounds__(TOY_THREADS) k_toy_delta(ToyParams P, ToyDelta D, uint64_t outer,
                                                           unsigned long long *hist) {
    const uint32_t p = toy_prime(P), R = p - P.kappa - 1;
    const uint32_t lane = threadIdx.x & 31;
    const uint64_t nw = (uint64_t)gridDim.x * (blockDim.x / 32);
    const uint32_t step = (uint32_t)((32ull * D.d[0]) % p);
    for (uint64_t o = (uint64_t)blockIdx.x * (blockDim.x / 32) + (threadIdx.x >> 5); o < outer; o += nw) {
        uint64_t base = 0, r = o;
        for (uint32_t i = 1; i < P.m; ++i) {
            base += (uint64_t)(1 + r % R) * D.d[i];
            r /= R;
        }
        uint32_t e = (uint32_t)((base + (uint64_t)(1 + lane) * D.d[0]) % p);
        for (uint32_t a1 = 1 + lane; a1 <= R; a1 += 32) {
            atomicAdd(&hist[e], 1ull);
            e += step;
            if (e >= p) e -= p;
        }
    }
}

}  // namespace pm
