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

// Both widths are computed on 32-bit limbs with explicit carry chains.

// Final step of Algorithm 2 (as read above) given v0 and v1 <= 2.
__device__ __forceinline__ Val alg2_finish(uint64_t v0, uint32_t v1, uint32_t k, int n) {
    const uint64_t kv1 = (uint64_t)(k * v1);
    const bool first = kv1 <= v0, second = v1 == 1;
    Val z;
    if (n == 32) {
        // values fit in lo: v0 - k v1, v0 + 2^32 or v0 + 2^32 - k
        const uint64_t add = first ? 0 : (second ? (1ull << 32) : (1ull << 32) - k);
        z.lo = v0 - (first ? kv1 : 0) + add;
        z.hi = 0;
    } else {
        // v0 - k v1, v0 + 2^64 or v0 + 2^64 - k (v0 < 2k in the last case)
        z.lo = v0 - (first ? kv1 : (second ? 0 : (uint64_t)k));
        z.hi = first ? 0 : (second ? 1 : (v0 >= k ? 1 : 0));
    }
    return z;
}

// n = 32: S = r0 + 2^32 r1 + 2^64 r2 (r2 <= 2^7 for the sums of Sec. 6.2).
__device__ __forceinline__ Val reduce32_limbs(uint32_t r0, uint32_t r1, uint32_t r2) {
    constexpr uint32_t k = (uint32_t)Fam<32>::K;
    const uint64_t u = (uint64_t)k * r1;  // k w1 = u0 + 2^32 u1
    const uint32_t u0 = (uint32_t)u, u1 = (uint32_t)(u >> 32);
    const uint32_t A = k * k * r2 + k * u1 + k;  // < 2^16
    // T = (r0 + A) - u0 + 2^32 = v0 + 2^32 v1
    uint32_t t0, c1, v0, bw;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, 0, 0;" : "=r"(t0), "=r"(c1) : "r"(r0), "r"(A));
    asm("sub.cc.u32 %0, %2, %3;\n\tsubc.u32 %1, 0, 0;" : "=r"(v0), "=r"(bw) : "r"(t0), "r"(u0));
    return alg2_finish(v0, 1u + c1 + bw, k, 32);  // bw = -borrow
}

// n = 64: S = (r1:r0) + 2^64 (r3:r2) + 2^128 r4.
__device__ __forceinline__ Val reduce64_limbs(uint32_t r0, uint32_t r1, uint32_t r2, uint32_t r3,
                                              uint32_t r4) {
    constexpr uint32_t k = (uint32_t)Fam<64>::K;
    // k w1 = u0 + 2^64 u1 with w1 = r3:r2
    const uint64_t p0 = (uint64_t)k * r2, p1 = (uint64_t)k * r3;
    uint32_t u0h, u1;
    asm("add.cc.u32 %0, %2, %3;\n\taddc.u32 %1, %4, 0;"
        : "=r"(u0h), "=r"(u1)
        : "r"((uint32_t)(p0 >> 32)), "r"((uint32_t)p1), "r"((uint32_t)(p1 >> 32)));
    const uint32_t u0l = (uint32_t)p0;
    const uint32_t A = k * k * r4 + k * u1 + k;  // < 2^32 for r4 < 2^24
    // T = (w0 + A) - u0 + 2^64 = v0 + 2^64 v1
    uint32_t t0, t1, c1, v0l, v0h, bw;
    asm("add.cc.u32 %0, %3, %4;\n\taddc.cc.u32 %1, %5, 0;\n\taddc.u32 %2, 0, 0;"
        : "=r"(t0), "=r"(t1), "=r"(c1)
        : "r"(r0), "r"(A), "r"(r1));
    asm("sub.cc.u32 %0, %3, %4;\n\tsubc.cc.u32 %1, %5, %6;\n\tsubc.u32 %2, 0, 0;"
        : "=r"(v0l), "=r"(v0h), "=r"(bw)
        : "r"(t0), "r"(u0l), "r"(t1), "r"(u0h));
    return alg2_finish(((uint64_t)v0h << 32) | v0l, 1u + c1 + bw, k, 64);
}

// n = 32: S = lo64 + 2^64 * w2 (w0, w1 are the 32-bit halves of lo64).
__device__ __forceinline__ uint64_t reduce32(uint64_t lo64, uint64_t w2) {
    return reduce32_limbs((uint32_t)lo64, (uint32_t)(lo64 >> 32), (uint32_t)w2).lo;
}

// n = 64: S = w0 + 2^64 w1 + 2^128 w2.
__device__ __forceinline__ Val reduce64(uint64_t w0, uint64_t w1, uint64_t w2) {
    return reduce64_limbs((uint32_t)w0, (uint32_t)(w0 >> 32), (uint32_t)w1, (uint32_t)(w1 >> 32),
                          (uint32_t)w2);
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

__device__ __forceinline__ uint32_t lo32(uint64_t x) { return (uint32_t)x; }
__device__ __forceinline__ uint32_t hi32(uint64_t x) { return (uint32_t)(x >> 32); }

// r += t on five 32-bit limbs.
__device__ __forceinline__ void add_limbs5(uint32_t (&r)[5], uint32_t t0, uint32_t t1, uint32_t t2,
                                           uint32_t t3, uint32_t t4) {
    asm("add.cc.u32 %0, %0, %5;\n\t"
        "addc.cc.u32 %1, %1, %6;\n\t"
        "addc.cc.u32 %2, %2, %7;\n\t"
        "addc.cc.u32 %3, %3, %8;\n\t"
        "addc.u32 %4, %4, %9;"
        : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4])
        : "r"(t0), "r"(t1), "r"(t2), "r"(t3), "r"(t4));
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
    // (b + sum) mod p, the sum formed on 32-bit limbs (L, H < 2^55, b < 2^32).
    __device__ __forceinline__ Val finish(uint64_t b) const {
        const uint32_t h0 = lo32(H) << 16, h1 = __funnelshift_l(lo32(H), hi32(H), 16), h2 = hi32(H) >> 16;
        uint32_t r0, r1, r2;
        asm("add.cc.u32 %0, %3, %4;\n\t"
            "addc.cc.u32 %1, %5, %6;\n\t"
            "addc.u32 %2, %7, 0;\n\t"
            "add.cc.u32 %0, %0, %8;\n\t"
            "addc.cc.u32 %1, %1, 0;\n\t"
            "addc.u32 %2, %2, 0;"
            : "=&r"(r0), "=&r"(r1), "=&r"(r2)
            : "r"(lo32(L)), "r"(h0), "r"(hi32(L)), "r"(h1), "r"(h2), "r"(lo32(b)));
        return reduce32_limbs(r0, r1, r2);
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
    // (b + sum) mod p, the sum formed on 32-bit limbs (every a_tu < 2^64,
    // a_2u < 2^53).
    __device__ __forceinline__ Val finish(uint64_t b) const {
        uint32_t r[5];
        asm("add.cc.u32 %0, %5, %6;\n\t"
            "addc.cc.u32 %1, %7, %8;\n\t"
            "addc.u32 %2, 0, 0;\n\t"
            "add.cc.u32 %1, %1, %9;\n\t"
            "addc.cc.u32 %2, %2, %10;\n\t"
            "addc.u32 %3, 0, 0;\n\t"
            "mov.u32 %4, 0;"
            : "=&r"(r[0]), "=&r"(r[1]), "=&r"(r[2]), "=&r"(r[3]), "=&r"(r[4])
            : "r"(lo32(b)), "r"(lo32(a00)), "r"(hi32(b)), "r"(hi32(a00)), "r"(lo32(a01)), "r"(hi32(a01)));
        add_limbs5(r, lo32(a10) << 25, __funnelshift_l(lo32(a10), hi32(a10), 25), hi32(a10) >> 7, 0, 0);
        add_limbs5(r, 0, lo32(a11) << 25, __funnelshift_l(lo32(a11), hi32(a11), 25), hi32(a11) >> 7, 0);
        add_limbs5(r, 0, lo32(a20) << 18, __funnelshift_l(lo32(a20), hi32(a20), 18), hi32(a20) >> 14, 0);
        add_limbs5(r, 0, 0, lo32(a21) << 18, __funnelshift_l(lo32(a21), hi32(a21), 18), hi32(a21) >> 14);
        return reduce64_limbs(r[0], r[1], r[2], r[3], r[4]);
    }
};

// --------------------------------------------------------------------------
// Carry-chain accumulators: the exact sum of full 32 x 32 -> 64 products
// kept on 32-bit limbs with the extended-precision multiply-adds of PTX
// (mad.lo.cc / madc.hi.cc / addc). One product costs a low and a high 32-bit
// multiply-add instead of the two 32 x 32 -> 64 multiply-adds of a split key,
// which halves the load on the multiply pipe (the key words stay whole).
// --------------------------------------------------------------------------

// n = 32: sum a*s on three limbs (128 products of two 32-bit words stay
// below 2^71).
struct AccC32 {
    uint32_t r0, r1, r2;
    __device__ __forceinline__ void zero() { r0 = r1 = r2 = 0; }
    __device__ __forceinline__ void add(uint32_t a, uint32_t s) {
        asm("mad.lo.cc.u32 %0, %3, %4, %0;\n\t"
            "madc.hi.cc.u32 %1, %3, %4, %1;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(r0), "+r"(r1), "+r"(r2)
            : "r"(a), "r"(s));
    }
    __device__ __forceinline__ void merge(const AccC32 &o) {
        asm("add.cc.u32 %0, %0, %3;\n\t"
            "addc.cc.u32 %1, %1, %4;\n\t"
            "addc.u32 %2, %2, %5;"
            : "+r"(r0), "+r"(r1), "+r"(r2)
            : "r"(o.r0), "r"(o.r1), "r"(o.r2));
    }
    // (b + sum) mod p, b < 2^32.
    __device__ __forceinline__ Val finish(uint64_t b) const {
        uint32_t t0, t1, t2;
        asm("add.cc.u32 %0, %3, %6;\n\t"
            "addc.cc.u32 %1, %4, 0;\n\t"
            "addc.u32 %2, %5, 0;"
            : "=r"(t0), "=r"(t1), "=r"(t2)
            : "r"(r0), "r"(r1), "r"(r2), "r"((uint32_t)b));
        return reduce32_limbs(t0, t1, t2);
    }
};

// n = 64: a * s = a0 s0 + 2^32 (a0 s1 + a1 s0) + 2^64 a1 s1 for the 32-bit
// halves. The straight terms a0 s0 + 2^64 a1 s1 go to five limbs (the sum of
// 128 products stays below 2^135), the cross terms to three limbs of their
// own (below 2^72), added in at the end with a 32-bit shift.
struct AccC64 {
    uint32_t r0, r1, r2, r3, r4;  // straight terms
    uint32_t x0, x1, x2;          // cross terms
    __device__ __forceinline__ void zero() { r0 = r1 = r2 = r3 = r4 = x0 = x1 = x2 = 0; }
    __device__ __forceinline__ void add(uint64_t a, uint64_t s) {
        const uint32_t a0 = (uint32_t)a, a1 = (uint32_t)(a >> 32), s0 = (uint32_t)s, s1 = (uint32_t)(s >> 32);
        asm("mad.lo.cc.u32 %0, %5, %7, %0;\n\t"
            "madc.hi.cc.u32 %1, %5, %7, %1;\n\t"
            "madc.lo.cc.u32 %2, %6, %8, %2;\n\t"
            "madc.hi.cc.u32 %3, %6, %8, %3;\n\t"
            "addc.u32 %4, %4, 0;"
            : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4)
            : "r"(a0), "r"(a1), "r"(s0), "r"(s1));
        asm("mad.lo.cc.u32 %0, %3, %6, %0;\n\t"
            "madc.hi.cc.u32 %1, %3, %6, %1;\n\t"
            "addc.u32 %2, %2, 0;\n\t"
            "mad.lo.cc.u32 %0, %4, %5, %0;\n\t"
            "madc.hi.cc.u32 %1, %4, %5, %1;\n\t"
            "addc.u32 %2, %2, 0;"
            : "+r"(x0), "+r"(x1), "+r"(x2)
            : "r"(a0), "r"(a1), "r"(s0), "r"(s1));
    }
    __device__ __forceinline__ void merge(const AccC64 &o) {
        asm("add.cc.u32 %0, %0, %5;\n\t"
            "addc.cc.u32 %1, %1, %6;\n\t"
            "addc.cc.u32 %2, %2, %7;\n\t"
            "addc.cc.u32 %3, %3, %8;\n\t"
            "addc.u32 %4, %4, %9;"
            : "+r"(r0), "+r"(r1), "+r"(r2), "+r"(r3), "+r"(r4)
            : "r"(o.r0), "r"(o.r1), "r"(o.r2), "r"(o.r3), "r"(o.r4));
        asm("add.cc.u32 %0, %0, %3;\n\t"
            "addc.cc.u32 %1, %1, %4;\n\t"
            "addc.u32 %2, %2, %5;"
            : "+r"(x0), "+r"(x1), "+r"(x2)
            : "r"(o.x0), "r"(o.x1), "r"(o.x2));
    }
    // (b + sum) mod p.
    __device__ __forceinline__ Val finish(uint64_t b) const {
        uint32_t t[5] = {r0, r1, r2, r3, r4};
        add_limbs5(t, (uint32_t)b, (uint32_t)(b >> 32), 0, 0, 0);
        add_limbs5(t, 0, x0, x1, x2, 0);
        return reduce64_limbs(t[0], t[1], t[2], t[3], t[4]);
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
