// pm_check.cuh -- exhaustive device checks of the 32-bit reduction and output
// step (property tests; the paper has no such entry points).
//
// The device code of Sec. 6.2 and Algorithm 2 (n = 32) and the 32-bit mixer
// of Sec. 7 take 32-bit inputs, so they can be checked on every input:
//   k_check_alg2_32    Algorithm 2 as the library reads it (alg2_finish) for
//                      every v0 < 2^32 and v1 <= 2, against (v0 + 2^32 v1)
//                      mod p formed by the integer remainder;
//   k_check_reduce32   the whole reduction (reduce32_limbs) of S = r0 +
//                      2^32 r1 + 2^64 r2 for every r0 < 2^32 and given
//                      (r1, r2), against S mod p = (r0 + r1 (2^32 mod p) +
//                      r2 (2^64 mod p)) mod p with 2^32 = p - 15 and
//                      2^64 = 225 (mod p), formed by the integer remainder;
//   k_check_mix32      mix32 followed by its inverse (the xorshift by 16
//                      undone by itself, the odd multiplier by its inverse
//                      mod 2^32 supplied by the caller, the xorshift by 13 by
//                      x = y ^ (y >> 13) ^ (y >> 26)) for every input: the
//                      mixer is a bijection iff nothing fails.
// Each counts its failures into *bad (warp-aggregated atomics).
//
// k_wait_probe exercises the failure path of the bounded waits instead: one
// warp waits on an mbarrier that expects an arrival nobody makes.
#pragma once
#include "pm_async.cuh"
#include "pm_device.cuh"

namespace pm {

constexpr int CHECK_MAX_PAIRS = 32;

struct CheckPairs {
    uint32_t r1[CHECK_MAX_PAIRS], r2[CHECK_MAX_PAIRS];
    int n;
};

__device__ __forceinline__ void count_bad(unsigned long long *bad, unsigned long long c) {
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) c += __shfl_down_sync(0xffffffffu, c, d);
    if ((threadIdx.x & 31) == 0 && c) atomicAdd(bad, c);
}

__global__ void __launch_bounds__(256) k_check_alg2_32(unsigned long long *bad) {
    constexpr uint64_t p = (1ull << 32) + 15;
    unsigned long long c = 0;
    const uint64_t total = 3ull << 32, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        const uint32_t v1 = (uint32_t)(x >> 32);
        const uint64_t v0 = x & 0xffffffffull;
        const Val z = alg2_finish(v0, v1, 15u, 32);
        c += z.hi != 0 || z.lo != (v0 + ((uint64_t)v1 << 32)) % p;
    }
    count_bad(bad, c);
}

__global__ void __launch_bounds__(256) k_check_reduce32(const CheckPairs P, unsigned long long *bad) {
    constexpr uint64_t p = (1ull << 32) + 15;
    unsigned long long c = 0;
    const uint64_t total = (uint64_t)P.n << 32, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        const int j = (int)(x >> 32);
        const uint32_t r0 = (uint32_t)x, r1 = P.r1[j], r2 = P.r2[j];
        const Val z = reduce32_limbs(r0, r1, r2);
        const uint64_t want = ((uint64_t)r1 * (p - 15) % p + r0 + (uint64_t)r2 * 225) % p;
        c += z.hi != 0 || z.lo != want;
    }
    count_bad(bad, c);
}

__global__ void __launch_bounds__(256) k_check_mix32(uint32_t ainv, unsigned long long *bad) {
    unsigned long long c = 0;
    const uint64_t total = 1ull << 32, stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t x = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; x < total; x += stride) {
        uint32_t y = mix32((uint32_t)x);
        y ^= y >> 16;
        y *= ainv;
        y = y ^ (y >> 13) ^ (y >> 26);
        c += y != (uint32_t)x;
    }
    count_bad(bad, c);
}

// The wait of mbar_wait (the one the TMA pipelines use) on a phase that never
// completes: it gives up after WAIT_LIMIT_NS, records PMP_ETIMEOUT in the
// device status word and raises the block's abort flag; the kernel then
// returns normally. *result = 1 if the wait reported success (it must not).
__global__ void k_wait_probe(int *result) {
    __shared__ __align__(8) uint64_t bar;
    __shared__ int abort_flag;
    if (threadIdx.x == 0) {
        mbar_init(&bar, 1);
        abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();
    const bool ok = mbar_wait(&bar, 0, &abort_flag);
    if (threadIdx.x == 0) *result = ok ? 1 : 0;
}

}  // namespace pm
