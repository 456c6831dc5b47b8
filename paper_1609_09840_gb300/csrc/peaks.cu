// peaks.cu -- microbenchmarks for the roofline denominators of the PM+ kernels:
// read-only HBM streaming bandwidth and the throughput of the integer
// multiplies the chunk sums are made of (32x32->64 multiply-add, 64-bit
// high multiply). Built as its own small library (libpmppeaks.so); the
// hashing library does not depend on it.
#include <cuda_runtime.h>

#include <cstdint>

namespace {

// Every thread XORs the 16-byte words it reads; the sink is written only if
// the accumulated value matches an impossible-to-predict key, which keeps the
// loads alive without adding stores.
__global__ void __launch_bounds__(256) k_read_stream(const uint4 *__restrict__ p, size_t n16,
                                                     uint32_t key, uint4 *sink) {
    uint4 acc = make_uint4(0, 0, 0, 0);
    const size_t stride = (size_t)gridDim.x * blockDim.x;
    size_t i = (size_t)blockIdx.x * blockDim.x + threadIdx.x;
    for (; i + 3 * stride < n16; i += 4 * stride) {
        const uint4 a = __ldcs(p + i), b = __ldcs(p + i + stride), c = __ldcs(p + i + 2 * stride),
                    d = __ldcs(p + i + 3 * stride);
        acc.x ^= a.x ^ b.x ^ c.x ^ d.x;
        acc.y ^= a.y ^ b.y ^ c.y ^ d.y;
        acc.z ^= a.z ^ b.z ^ c.z ^ d.z;
        acc.w ^= a.w ^ b.w ^ c.w ^ d.w;
    }
    for (; i < n16; i += stride) {
        const uint4 a = __ldcs(p + i);
        acc.x ^= a.x;
        acc.y ^= a.y;
        acc.z ^= a.z;
        acc.w ^= a.w;
    }
    if ((acc.x ^ acc.y ^ acc.z ^ acc.w) == key) sink[0] = acc;
}

// 16 independent chains per thread of x = lo32(x) * a + x (one 32x32->64
// multiply-add each); the chains depend on themselves, so nothing is hoisted.
__global__ void __launch_bounds__(256) k_imad_wide(uint32_t a, int iters, uint64_t key,
                                                   uint64_t *sink) {
    uint64_t x[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) x[j] = (uint64_t)(threadIdx.x + 977u * j + blockIdx.x);
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j) x[j] += (uint64_t)(uint32_t)x[j] * a;
    }
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s ^= x[j];
    if (s == key) sink[0] = s;
}

// 8 independent chains of x = umulhi64(x, a) + x (one 64-bit high multiply).
__global__ void __launch_bounds__(256) k_mulhi64(uint64_t a, int iters, uint64_t key,
                                                 uint64_t *sink) {
    uint64_t x[8];
#pragma unroll
    for (int j = 0; j < 8; ++j) x[j] = (uint64_t)(threadIdx.x + 131u * j + blockIdx.x) * 0x9e3779b97f4a7c15ull;
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 8; ++j) x[j] += __umul64hi(x[j], a);
    }
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < 8; ++j) s ^= x[j];
    if (s == key) sink[0] = s;
}

// 16 independent carry chains per thread of one 32 x 32 product added to a
// three-limb accumulator (mad.lo.cc, madc.hi.cc, addc): the multiply-add of
// the single-buffer kernel. The next word depends on the low limb.
__global__ void __launch_bounds__(256) k_madc(uint32_t a, int iters, uint64_t key, uint64_t *sink) {
    uint32_t l0[16], l1[16], l2[16];
#pragma unroll
    for (int j = 0; j < 16; ++j) {
        l0[j] = threadIdx.x + 977u * j + blockIdx.x;
        l1[j] = 0;
        l2[j] = 0;
    }
    for (int i = 0; i < iters; ++i) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
            asm volatile("mad.lo.cc.u32 %0, %0, %3, %0;\n\tmadc.hi.cc.u32 %1, %0, %3, %1;\n\taddc.u32 %2, %2, 0;"
                         : "+r"(l0[j]), "+r"(l1[j]), "+r"(l2[j])
                         : "r"(a));
    }
    uint64_t s = 0;
#pragma unroll
    for (int j = 0; j < 16; ++j) s ^= l0[j] ^ ((uint64_t)l1[j] << 32) ^ l2[j];
    if (s == key) sink[0] = s;
}
int sms() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n;
}

// Time `reps` launches with CUDA events on the default stream, best of them.
template <class F>
float best_ms(F launch, int reps) {
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    for (int r = 0; r < reps; ++r) {
        cudaEventRecord(a);
        launch();
        cudaEventRecord(b);
        cudaEventSynchronize(b);
        float ms = 0;
        cudaEventElapsedTime(&ms, a, b);
        if (ms < best) best = ms;
    }
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    return best;
}

}  // namespace

extern "C" {

// Read-only stream over `bytes` (a multiple of 16) of the device buffer d_buf.
// Returns GB/s (1e9 bytes per second), best of `reps`, or a negative value on
// a CUDA error.
double pmpk_read_gbs(const void *d_buf, size_t bytes, void *d_sink, int reps) {
    const size_t n16 = bytes / 16;
    const int grid = sms() * 8;
    const float ms = best_ms([&] {
        k_read_stream<<<grid, 256>>>(static_cast<const uint4 *>(d_buf), n16, 0x9e3779b9u,
                                     static_cast<uint4 *>(d_sink));
    }, reps);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return (double)bytes / (ms * 1e-3) / 1e9;
}

// 32x32->64 multiply-adds per second (whole GPU).
double pmpk_imad_wide_per_s(void *d_sink, int reps) {
    const int grid = sms() * 8, iters = 4096;
    const float ms = best_ms([&] {
        k_imad_wide<<<grid, 256>>>(0x9e3779b9u, iters, 0x1234567ull, static_cast<uint64_t *>(d_sink));
    }, reps);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return (double)grid * 256 * iters * 16 / (ms * 1e-3);
}

// 64-bit high multiplies per second (whole GPU).
double pmpk_mulhi64_per_s(void *d_sink, int reps) {
    const int grid = sms() * 8, iters = 2048;
    const float ms = best_ms([&] {
        k_mulhi64<<<grid, 256>>>(0x9e3779b97f4a7c15ull, iters, 0x1234567ull,
                                 static_cast<uint64_t *>(d_sink));
    }, reps);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return (double)grid * 256 * iters * 8 / (ms * 1e-3);
}

// Full 32 x 32 products accumulated on carry chains (mad.lo.cc + madc.hi.cc
// + addc) per second (whole GPU).
double pmpk_madc_per_s(void *d_sink, int reps) {
    const int grid = sms() * 8, iters = 2048;
    const float ms = best_ms([&] {
        k_madc<<<grid, 256>>>(0x9e3779b9u, iters, 0x1234567ull, static_cast<uint64_t *>(d_sink));
    }, reps);
    if (cudaGetLastError() != cudaSuccess) return -1.0;
    return (double)grid * 256 * iters * 16 / (ms * 1e-3);
}

}  // extern "C"
