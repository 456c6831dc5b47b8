// pm_device.cuh -- integer arithmetic of PM+ hashing on the device (sm_103a).
//
// PM+-Multilinear (arXiv 1609.09840, Sec. 5, eq. 2wlinear):
//     f(s_1..s_m) = (b + sum_i a_i s_i) mod p,  p = 2^n + k,
// with the parameters of Table "parameters" (Sec. 6.1). The sum is formed
// exactly (three words, Sec. 6.2) and reduced once per chunk with the
// pseudo+Mersenne reduction of Sec. 6.2 followed by Algorithm 2.
#pragma once
#include <cstdint>

namespace pm {

constexpr int M = 128;          // words per chunk (Table "parameters")
constexpr int LMAX = 8;         // levels of the tree (Table "parameters")
constexpr int KEY_ROW = M + 1;  // b_j followed by a_{j,1..m}

template <int N> struct Fam;
template <> struct Fam<32> {
    static constexpr uint64_t K = 15;      // p = 2^32 + 15
    static constexpr uint64_t KAPPA = 28;  // a_i in (0, p - 28)
    typedef uint32_t word;
    static constexpr int W = 4;
};
template <> struct Fam<64> {
    static constexpr uint64_t K = 13;      // p = 2^64 + 13
    static constexpr uint64_t KAPPA = 24;  // a_i in (0, p - 24)
    typedef uint64_t word;
    static constexpr int W = 8;
};

// A value of [0, p): lo + 2^64 * hi, hi in {0, 1} (hi is always 0 for n = 32,
// whose values < 2^32 + 15 fit in lo).
struct Val {
    uint64_t lo, hi;
};

// Exact 192-bit unsigned integer w0 + 2^64 w1 + 2^128 w2.
struct U192 {
    uint64_t w0, w1, w2;
};

__device__ __forceinline__ void add192(U192 &a, uint64_t b0, uint64_t b1, uint64_t b2) {
    asm("add.cc.u64 %0, %0, %3;\n\t"
        "addc.cc.u64 %1, %1, %4;\n\t"
        "addc.u64 %2, %2, %5;"
        : "+l"(a.w0), "+l"(a.w1), "+l"(a.w2)
        : "l"(b0), "l"(b1), "l"(b2));
}

__device__ __forceinline__ void add192(U192 &a, const U192 &b) { add192(a, b.w0, b.w1, b.w2); }

// a += v * 2^sh for a compile-time shift 0 <= sh < 128.
template <int SH>
__device__ __forceinline__ void add_shifted(U192 &a, uint64_t v) {
    if constexpr (SH == 0) {
        add192(a, v, 0, 0);
    } else if constexpr (SH < 64) {
        add192(a, v << SH, v >> (64 - SH), 0);
    } else if constexpr (SH == 64) {
        add192(a, 0, v, 0);
    } else {
        add192(a, 0, v << (SH - 64), v >> (128 - SH));
    }
}

__device__ __forceinline__ U192 shfl_down192(const U192 &x, int d) {
    U192 y;
    y.w0 = __shfl_down_sync(0xffffffffu, x.w0, d);
    y.w1 = __shfl_down_sync(0xffffffffu, x.w1, d);
    y.w2 = __shfl_down_sync(0xffffffffu, x.w2, d);
    return y;
}

// Sum of x over the 32 lanes of a warp, result in lane 0.
__device__ __forceinline__ U192 warp_sum192(U192 x) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) add192(x, shfl_down192(x, d));
    return x;
}

// Product a * s of a key word a < p - kappa and a level value s < p. By the
// choice of kappa (Sec. 6.1) the product is below 2^{2n}.
__device__ __forceinline__ void mac(U192 &acc, uint32_t a, const Val &s) {
    // n = 32: s < 2^32 + 15, a < 2^32 - 13, so a*s < 2^64.
    add192(acc, (uint64_t)a * s.lo, 0, 0);
}
__device__ __forceinline__ void mac(U192 &acc, uint64_t a, const Val &s) {
    // n = 64: a*s = a*lo + 2^64 * (hi ? a : 0) < 2^128.
    uint64_t lo = a * s.lo;
    uint64_t hi = __umul64hi(a, s.lo) + (s.hi ? a : 0);
    add192(acc, lo, hi, 0);
}

// --------------------------------------------------------------------------
// Reduction modulo p = 2^n + k of a three-word sum (Sec. 6.2).
//   S = w0 + 2^n w1 + 2^{2n} w2  ==  w0 - k w1 + k^2 w2  (mod p).
// With k w1 = u0 + 2^n u1:
//   S == (w0 + k^2 w2 + k u1) + (2^n + k - u0)  (mod p),
// a two-word value v0 + 2^n v1 with v1 <= 2 (the bound of Sec. 6.2 for
// w2 <= m), finished by Algorithm 2. Reading of Algorithm 2 (its printed
// listing swaps the names of the two inputs and ends with "v0 - k"): with
// input v0 + 2^n v1,
//   if k v1 <= v0:      return v0 - k v1
//   else if v1 == 1:    return v0 + 2^n
//   else (v1 == 2):     return v0 + 2^n - k      (2 * 2^n == 2^n - k mod p)
// which lies in [0, p) in every branch.
// --------------------------------------------------------------------------

// n = 32: S = lo64 + 2^64 * w2 (w0, w1 are the 32-bit halves of lo64).
__device__ __forceinline__ uint64_t reduce32(uint64_t lo64, uint64_t w2) {
    const uint64_t k = Fam<32>::K;
    const uint64_t w0 = lo64 & 0xffffffffull, w1 = lo64 >> 32;
    const uint64_t u = k * w1;
    const uint64_t u0 = u & 0xffffffffull, u1 = u >> 32;
    const uint64_t T = w0 + k * k * w2 + k * u1 + ((1ull << 32) + k - u0);
    const uint64_t v0 = T & 0xffffffffull, v1 = T >> 32;
    if (k * v1 <= v0) return v0 - k * v1;
    if (v1 == 1) return v0 + (1ull << 32);
    return v0 + (1ull << 32) - k;
}

// n = 64: S = w0 + 2^64 w1 + 2^128 w2.
__device__ __forceinline__ Val reduce64(uint64_t w0, uint64_t w1, uint64_t w2) {
    const uint64_t k = Fam<64>::K;
    const uint64_t u0 = k * w1;              // low word of k * w1
    const uint64_t u1 = __umul64hi(k, w1);   // high word, < k
    // T = (w0 + k^2 w2 + k u1) + (2^64 + k - u0)
    unsigned __int128 T = (unsigned __int128)w0 + (unsigned __int128)(k * k * w2 + k * u1);
    T += ((unsigned __int128)1 << 64) + k;
    T -= u0;
    const uint64_t v0 = (uint64_t)T, v1 = (uint64_t)(T >> 64);
    Val z;
    if (k * v1 <= v0) {
        z.lo = v0 - k * v1;
        z.hi = 0;
    } else if (v1 == 1) {
        z.lo = v0;
        z.hi = 1;
    } else {
        z.lo = v0 - k;  // v0 + 2^64 - k, with v0 < 2k
        z.hi = v0 >= k ? 1 : 0;
    }
    return z;
}

template <int N> __device__ __forceinline__ Val reduce(const U192 &S);
template <> __device__ __forceinline__ Val reduce<32>(const U192 &S) {
    Val z;
    z.lo = reduce32(S.w0, S.w1);
    z.hi = 0;
    return z;
}
template <> __device__ __forceinline__ Val reduce<64>(const U192 &S) {
    return reduce64(S.w0, S.w1, S.w2);
}

// --------------------------------------------------------------------------
// Output step: z = h mod 2^n (Sec. 5, end), then the mixer of Sec. 7.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint32_t mix32(uint32_t z) {
    z ^= z >> 13;
    z *= 0xab3be54fu;
    z ^= z >> 16;
    return z;
}
__device__ __forceinline__ uint64_t mix64(uint64_t z) {
    z ^= z >> 33;
    z *= 0xc4ceb9fe1a85ec53ull;
    z ^= z >> 33;
    return z;
}

// --------------------------------------------------------------------------
// Key words split for carry-free multiply-accumulate in the hot loops.
// n = 32: a = aL + 2^16 aH with aL, aH < 2^16; a 128-word sum of aL * s
//   (s < 2^32) stays below 2^55, so two 64-bit accumulators never carry.
// n = 64: a = a0 + 2^25 a1 + 2^50 a2 with a0, a1 < 2^25, a2 < 2^14, and
//   s = s0 + 2^32 s1; each of the six 128-term sums a_t * s_u stays
//   below 128 * 2^57 = 2^64.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint2 split_key32(uint32_t a) { return make_uint2(a & 0xffffu, a >> 16); }
__device__ __forceinline__ uint4 split_key64(uint64_t a) {
    return make_uint4((uint32_t)(a & 0x1ffffffull), (uint32_t)((a >> 25) & 0x1ffffffull),
                      (uint32_t)(a >> 50), 0u);
}

struct Acc32 {  // sum a*s = L + 2^16 H
    uint64_t L, H;
    __device__ __forceinline__ void zero() { L = H = 0; }
    __device__ __forceinline__ void add(uint2 k, uint32_t s) {
        L += (uint64_t)k.x * s;
        H += (uint64_t)k.y * s;
    }
    __device__ __forceinline__ void merge(const Acc32 &o) {
        L += o.L;
        H += o.H;
    }
    // b + sum, exactly.
    __device__ __forceinline__ U192 total(uint64_t b) const {
        U192 S = {b, 0, 0};
        add_shifted<0>(S, L);
        add_shifted<16>(S, H);
        return S;
    }
};

struct Acc64 {  // sum a*s = sum_{t,u} A[t][u] 2^{25 t + 32 u}
    uint64_t a00, a01, a10, a11, a20, a21;
    __device__ __forceinline__ void zero() { a00 = a01 = a10 = a11 = a20 = a21 = 0; }
    __device__ __forceinline__ void add(uint4 k, uint64_t s) {
        const uint32_t s0 = (uint32_t)s, s1 = (uint32_t)(s >> 32);
        a00 += (uint64_t)k.x * s0;
        a01 += (uint64_t)k.x * s1;
        a10 += (uint64_t)k.y * s0;
        a11 += (uint64_t)k.y * s1;
        a20 += (uint64_t)k.z * s0;
        a21 += (uint64_t)k.z * s1;
    }
    __device__ __forceinline__ void merge(const Acc64 &o) {
        a00 += o.a00;
        a01 += o.a01;
        a10 += o.a10;
        a11 += o.a11;
        a20 += o.a20;
        a21 += o.a21;
    }
    __device__ __forceinline__ U192 total(uint64_t b) const {
        U192 S = {b, 0, 0};
        add_shifted<0>(S, a00);
        add_shifted<32>(S, a01);
        add_shifted<25>(S, a10);
        add_shifted<57>(S, a11);
        add_shifted<50>(S, a20);
        add_shifted<82>(S, a21);
        return S;
    }
};

// --------------------------------------------------------------------------
// splitmix64 (Steele, Lea, Flood 2014) for key expansion.
// --------------------------------------------------------------------------
__device__ __forceinline__ uint64_t splitmix64_at(uint64_t seed, uint64_t i) {
    uint64_t z = seed + (i + 1) * 0x9e3779b97f4a7c15ull;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}

}  // namespace pm
