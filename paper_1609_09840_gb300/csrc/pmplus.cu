// pmplus.cu -- C ABI of the PM+ hashing library (see include/pmplus.h).
#include <cuda.h>
#include <cuda_runtime.h>
#include <cudaTypedefs.h>

#include <cstdio>
#include <cstring>
#include <mutex>
#include <utility>

#include "../../include/pmplus.h"
#include "pm_kernels.cuh"
#include "pm_tree.cuh"
#include "pm_lane.cuh"
#include "pm_range.cuh"
#include "pm_stream.cuh"
#include "pm_fixed.cuh"
#include "pm_collide.cuh"
#include "pm_toy.cuh"
#include "pm_check.cuh"

using namespace pm;

struct pmp_key {
    int width;
    int device;
    void *d_words;  // LMAX * KEY_ROW words of width/8 bytes
    // host copies of what kernels take as launch parameters: b_1 and the
    // split level-1 key words of every 8-byte unit of a chunk
    uint64_t b1;
    uint4 k1[M];
};

namespace {

constexpr int MAX_DEVICES = 64;
constexpr int TREE_STAGE_CHOICES[4] = {2, 3, 4, 6};

// Tuning knobs (process-wide). Staging depth of the tree kernel per width.
int g_tree_stages[2] = {4, 4};  // [width == 64]
int g_batch_p1 = 6;           // PMP_KNOB_BATCH_P1 (units of pass 1 of the batch tile kernel)
int g_batch_sched = PMP_BATCH_SORTED;  // PMP_KNOB_BATCH_SCHED (schedule of one-chunk strings)
int g_chunk_stages[2] = {2, 2};        // PMP_KNOB_CHUNK_STAGES_32/64 (staging depth of the chunk kernel)
int g_stream_segment = 1 << 19;        // PMP_KNOB_STREAM_SEGMENT (level-1 chunks per update segment)
int g_batch_range = 1024;              // PMP_KNOB_BATCH_RANGE (strings per range of the sorted schedule)

size_t key_bytes(int width) { return (size_t)LMAX * KEY_ROW * (size_t)(width / 8); }

int cuda_fail(cudaError_t e) {
    if (e == cudaSuccess) return PMP_OK;
    (void)cudaGetLastError();  // clear a non-sticky error
    return PMP_ECUDA;
}

// cuTensorMapEncodeTiled through the runtime's driver entry point, so the
// library does not link libcuda directly.
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static std::once_flag once;
    std::call_once(once, [] {
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    });
    return fn;
}

struct DeviceInfo {
    int sms = 0;
    int tree_blocks_per_sm[2][4] = {{0}};  // [width == 64][stage choice]
    int lane_blocks_per_sm[2][2] = {{0, 0}, {0, 0}};  // [width == 64][p1 == 8]
    int range_blocks_per_sm[2][2] = {{0, 0}, {0, 0}};  // [width == 64][1024 strings a range]
    int chunk_blocks_per_sm[2][2] = {{0, 0}, {0, 0}};  // [width == 64][3 stages]
    int fixed_blocks_per_sm[2][6] = {};  // [width == 64][long; 3..5, 1, 2, 6..9 units; 6..9 by 16-byte loads]
    bool ready = false;
};
DeviceInfo g_dev[MAX_DEVICES];
std::mutex g_dev_mu;

int stage_index(int stages) {
    for (int i = 0; i < 4; ++i)
        if (TREE_STAGE_CHOICES[i] == stages) return i;
    return -1;
}

template <int N, int S>
int tree_setup_one(DeviceInfo &d) {
    const size_t smem = TreeSmem<N, S>::ALLOC;
    cudaError_t e =
        cudaFuncSetAttribute(k_tree<N, S>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return cuda_fail(e);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_tree<N, S>, TREE_THREADS, smem);
    if (e != cudaSuccess) return cuda_fail(e);
    d.tree_blocks_per_sm[N == 64][stage_index(S)] = nb > 0 ? nb : 1;
    return PMP_OK;
}

template <int N, int S>
int chunk_setup(int &blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_long_chunk<N, S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)chunk_smem_bytes<N, S>());
    if (e != cudaSuccess) return cuda_fail(e);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_long_chunk<N, S>, LC_THREADS, chunk_smem_bytes<N, S>());
    if (e != cudaSuccess) return cuda_fail(e);
    blocks_per_sm = nb > 0 ? nb : 1;
    return PMP_OK;
}

template <int N, class C>
int range_setup(int &blocks_per_sm) {
    cudaError_t e = cudaFuncSetAttribute(k_batch_range<N, C>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)range_smem_bytes<N, C>());
    if (e != cudaSuccess) return cuda_fail(e);
    int nb = 0;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_range<N, C>, C::THREADS, range_smem_bytes<N, C>());
    if (e != cudaSuccess) return cuda_fail(e);
    blocks_per_sm = nb > 0 ? nb : 1;
    return PMP_OK;
}

template <int N>
int batch_setup(DeviceInfo &d) {
    int nb = 0, rc = PMP_OK;
    cudaError_t e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_lane<N, 6>, BL_THREADS, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.lane_blocks_per_sm[N == 64][0] = nb > 0 ? nb : 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_batch_lane<N, 8>, BL_THREADS, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.lane_blocks_per_sm[N == 64][1] = nb > 0 ? nb : 1;
    rc = range_setup<N, RangeNarrow>(d.range_blocks_per_sm[N == 64][0]);
    if (rc) return rc;
    rc = range_setup<N, RangeWide>(d.range_blocks_per_sm[N == 64][1]);
    if (rc) return rc;
    rc = chunk_setup<N, 2>(d.chunk_blocks_per_sm[N == 64][0]);
    if (rc) return rc;
    rc = chunk_setup<N, 3>(d.chunk_blocks_per_sm[N == 64][1]);
    if (rc) return rc;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fixed<N>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.fixed_blocks_per_sm[N == 64][0] = nb > 0 ? nb : 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fixed_few<N, 5, false>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.fixed_blocks_per_sm[N == 64][1] = nb > 0 ? nb : 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fixed_few<N, 2, false>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.fixed_blocks_per_sm[N == 64][3] = nb > 0 ? nb : 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fixed_few<N, FIXED_FEW_MAX, false>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.fixed_blocks_per_sm[N == 64][4] = nb > 0 ? nb : 1;
    // one key per thread: fewer registers, more resident blocks
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fixed_few<N, FIXED_FEW_MAX, true>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.fixed_blocks_per_sm[N == 64][5] = nb > 0 ? nb : 1;
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&nb, k_fixed_one<N>, 256, 0);
    if (e != cudaSuccess) return cuda_fail(e);
    d.fixed_blocks_per_sm[N == 64][2] = nb > 0 ? nb : 1;
    return PMP_OK;
}

template <int N>
int tree_setup(DeviceInfo &d) {
    int rc = tree_setup_one<N, 2>(d);
    if (!rc) rc = tree_setup_one<N, 3>(d);
    if (!rc) rc = tree_setup_one<N, 4>(d);
    if (!rc) rc = tree_setup_one<N, 6>(d);
    return rc;
}

int device_info(DeviceInfo **out) {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= MAX_DEVICES) return PMP_EINVAL;
    std::lock_guard<std::mutex> lk(g_dev_mu);
    DeviceInfo &d = g_dev[dev];
    if (!d.ready) {
        e = cudaDeviceGetAttribute(&d.sms, cudaDevAttrMultiProcessorCount, dev);
        if (e != cudaSuccess) return cuda_fail(e);
        int rc = tree_setup<32>(d);
        if (rc) return rc;
        rc = tree_setup<64>(d);
        if (rc) return rc;
        rc = batch_setup<32>(d);
        if (rc) return rc;
        rc = batch_setup<64>(d);
        if (rc) return rc;
        d.ready = true;
    }
    *out = &d;
    return PMP_OK;
}

// Level structure of Algorithm 1 for a string of `len` bytes.
struct Plan {
    uint64_t n0, F;
    uint64_t c[LMAX + 2];
    int levels;
    uint64_t ntiles;  // level-2 chunks = work items of the tree kernel
    size_t vals_off[LMAX + 2], ctr_off[LMAX + 2], tile_ctr_off;
    size_t ctr_begin, ctr_bytes, scratch;
};

int make_plan(int width, uint64_t len, Plan &P) {
    const uint64_t W = (uint64_t)width / 8;
    memset(&P, 0, sizeof P);
    P.n0 = len / W + 1;
    P.F = len / ((uint64_t)M * W);
    uint64_t c = P.n0;
    int lv = 0;
    do {
        c = (c + M - 1) / M;
        ++lv;
        if (lv > LMAX) return PMP_ETOOLONG;
        P.c[lv] = c;
    } while (c > 1);
    P.levels = lv;
    P.ntiles = lv >= 2 ? P.c[2] : 1;
    size_t off = 0;
    for (int j = 2; j < lv; ++j) {  // values produced by levels 2 .. levels-1
        P.vals_off[j] = off;
        off += sizeof(Val) * P.c[j];
    }
    off = (off + 255) / 256 * 256;
    P.ctr_begin = off;
    if (P.ntiles > 1) {  // device work counter of the tree kernel
        P.tile_ctr_off = off;
        off += 8;
    }
    for (int j = 3; j <= lv; ++j) {
        P.ctr_off[j] = off;
        off += sizeof(unsigned) * P.c[j];
    }
    P.ctr_bytes = off - P.ctr_begin;
    P.scratch = off;
    return PMP_OK;
}

// The tensor map of F whole level-1 chunks at d_buf (16-byte aligned): rows
// of m W bytes, boxes of 128 bytes x 128 rows, 128-byte swizzle.
template <int N>
int encode_chunk_map(const void *d_buf, uint64_t F, CUtensorMap &tmap) {
    // rows: whole chunks, or half chunks where the tree kernel reads those
    const uint64_t parts = half_rows<N>() ? 2 : 1;
    if (F * parts > 0x7fffffffull) return PMP_EINVAL;
    PFN_cuTensorMapEncodeTiled_v12000 enc = encode_fn();
    if (!enc) return PMP_ECUDA;
    const uint64_t row = (uint64_t)M * (N / 8) / parts;
    cuuint64_t dims[2] = {row, F * parts};
    cuuint64_t strides[1] = {row};
    cuuint32_t box[2] = {TILE_ROW_BYTES, TREE_CONSUMERS};
    cuuint32_t estr[2] = {1, 1};
    CUresult cr = enc(&tmap, CU_TENSOR_MAP_DATA_TYPE_UINT8, 2, const_cast<void *>(d_buf), dims, strides, box,
                      estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                      CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return cr == CUDA_SUCCESS ? PMP_OK : PMP_ECUDA;
}

// One launch of the tree kernel over `ntiles` tiles, at the tuned staging
// depth, one wave of resident blocks at most.
template <int N>
unsigned tree_grid(const DeviceInfo *dev, uint64_t ntiles) {
    const int si = stage_index(g_tree_stages[N == 64]);
    const uint64_t cap = (uint64_t)dev->sms * dev->tree_blocks_per_sm[N == 64][si];
    return (unsigned)(ntiles < cap ? ntiles : cap);
}

// A launch of the tree kernel at staging depth S; with `pdl`, as a
// programmatic dependent of the kernel before it on the stream (it may start
// once that kernel's blocks have all triggered; only a level-2 mode tree
// launch triggers before it ends, and this kernel reads nothing such a
// launch writes).
template <int N, int S>
cudaError_t launch_tree_at(const CUtensorMap &tmap, const TreeParams &tp, unsigned grid, bool pdl,
                           cudaStream_t stream) {
    if (!pdl) {
        k_tree<N, S><<<grid, TREE_THREADS, TreeSmem<N, S>::ALLOC, stream>>>(tmap, tp);
        return cudaGetLastError();
    }
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(TREE_THREADS);
    cfg.dynamicSmemBytes = TreeSmem<N, S>::ALLOC;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_tree<N, S>, tmap, tp);
}

template <int N>
int launch_tree(const DeviceInfo *dev, const CUtensorMap &tmap, const TreeParams &tp, uint64_t ntiles,
                cudaStream_t stream, bool pdl = false) {
    const int stages = g_tree_stages[N == 64];
    const unsigned grid = tree_grid<N>(dev, ntiles);
    cudaError_t e;
    switch (stages) {
        case 2: e = launch_tree_at<N, 2>(tmap, tp, grid, pdl, stream); break;
        case 3: e = launch_tree_at<N, 3>(tmap, tp, grid, pdl, stream); break;
        case 6: e = launch_tree_at<N, 6>(tmap, tp, grid, pdl, stream); break;
        default: e = launch_tree_at<N, 4>(tmap, tp, grid, pdl, stream); break;
    }
    return cuda_fail(e);
}

template <int N>
int hash_one(const pmp_key *key, const void *d_buf, uint64_t len, void *d_out, uint64_t *d_raw,
             void *d_scratch, size_t scratch_bytes, cudaStream_t stream) {
    if (!key || key->width != N || !d_out || (!d_buf && len)) return PMP_EINVAL;
    if (len && (reinterpret_cast<uintptr_t>(d_buf) & 15)) return PMP_EALIGN;
    Plan plan;
    int rc = make_plan(N, len, plan);
    if (rc) return rc;
    if (plan.scratch > scratch_bytes || (plan.scratch && !d_scratch)) return PMP_EINVAL;
    DeviceInfo *dev;
    rc = device_info(&dev);
    if (rc) return rc;

    TreeParams tp;
    memset(&tp, 0, sizeof tp);
    tp.buf = static_cast<const uint8_t *>(d_buf);
    tp.len = len;
    tp.F = plan.F;
    for (int j = 0; j < LMAX + 2; ++j) tp.c[j] = plan.c[j];
    tp.c[0] = plan.n0;
    tp.levels = plan.levels;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);
    for (int j = 2; j < plan.levels; ++j) tp.vals[j] = reinterpret_cast<Val *>(scr + plan.vals_off[j]);
    for (int j = 3; j <= plan.levels; ++j)
        tp.ctr[j] = reinterpret_cast<unsigned *>(scr + plan.ctr_off[j]);
    if (plan.ntiles > 1)
        tp.tile_ctr = reinterpret_cast<unsigned long long *>(scr + plan.tile_ctr_off);
    tp.key = key->d_words;
    tp.out = d_out;
    tp.raw = d_raw;

    CUtensorMap tmap;
    memset(&tmap, 0, sizeof tmap);
    if (plan.F > 0) {
        rc = encode_chunk_map<N>(d_buf, plan.F, tmap);
        if (rc) return rc;
        tp.use_tma = 1;
    }
    if (plan.ctr_bytes) {
        cudaError_t e = cudaMemsetAsync(scr + plan.ctr_begin, 0, plan.ctr_bytes, stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return launch_tree<N>(dev, tmap, tp, plan.ntiles, stream);
}

// Scratch of a batched call (width, data_bytes >= offsets[n]):
// [0, 256)    counters (work items reserved / claimed, tree storage)
// items       one per level-2 segment of the strings of at least BIG_CHUNKS
//             chunks: at most D + 2 data_bytes / (BIG_CHUNKS m W) + 2,
//             D = data_bytes / (m^2 W) + 1
// tree store  levels >= 2 of the strings of more than m chunks: at most 120 D
//             bytes
// Strings of fewer chunks need no scratch (the tile kernel hashes them).
struct BatchScratch {
    size_t big_str, big_pool, big_seg, pool, total;
    uint64_t big_cap, pool_cap;
};

BatchScratch batch_scratch(int width, uint64_t data_bytes) {
    BatchScratch b;
    const uint64_t W = (uint64_t)width / 8;
    const uint64_t D = data_bytes / ((uint64_t)M * M * W) + 1;
    auto up = [](size_t x) { return (x + 255) / 256 * 256; };
    b.big_cap = D + 2 * (data_bytes / (BIG_CHUNKS * M * W)) + 2;
    b.pool_cap = 120 * D;
    b.big_str = 256;
    b.big_pool = b.big_str + up(8 * b.big_cap);
    b.big_seg = b.big_pool + up(8 * b.big_cap);
    b.pool = b.big_seg + up(4 * b.big_cap);
    b.total = b.pool + up(b.pool_cap);
    return b;
}

// The sorted-range kernel: one block per range at most, one wave of resident blocks.
template <int N, class C>
void launch_range(const BatchParams &bp, int64_t n, int64_t resident, cudaStream_t stream) {
    const int64_t blocks = (n + C::RS - 1) / C::RS;
    const unsigned grid = (unsigned)(blocks < resident ? blocks : resident);
    k_batch_range<N, C><<<grid, C::THREADS, range_smem_bytes<N, C>(), stream>>>(bp);
}

// Launch of the chunk kernel as a programmatic dependent of the tile kernel
// on the same stream: its launch is processed while the tile kernel runs.
template <int N, int S>
cudaError_t launch_chunk_kernel(const BatchParams &bp, unsigned grid, cudaStream_t stream) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(LC_THREADS);
    cfg.dynamicSmemBytes = chunk_smem_bytes<N, S>();
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_long_chunk<N, S>, bp);
}

template <int N>
int hash_batch(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets, int64_t n,
               void *d_out, int raw, void *d_scratch, size_t scratch_bytes, cudaStream_t stream,
               int *d_status = nullptr) {
    if (!key || key->width != N || n < 0 || (n > 0 && (!d_offsets || !d_out || !d_base)))
        return PMP_EINVAL;
    if (n == 0) return PMP_OK;
    if (reinterpret_cast<uintptr_t>(d_base) & 15) return PMP_EALIGN;
    if (n > 0xffffffffll) return PMP_EINVAL;
    // the largest data size this scratch covers (the work lists grow with it)
    if (!d_scratch || scratch_bytes < batch_scratch(N, 0).total) return PMP_EINVAL;
    uint64_t lo = 0, hi = 1ull << 62;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        if (batch_scratch(N, mid).total <= scratch_bytes)
            lo = mid;
        else
            hi = mid - 1;
    }
    const BatchScratch bs = batch_scratch(N, lo);
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    uint8_t *scr = static_cast<uint8_t *>(d_scratch);
    BatchParams bp;
    memset(&bp, 0, sizeof bp);
    bp.base = d_base;
    bp.off = d_offsets;
    bp.n = n;
    bp.key = key->d_words;
    bp.out = d_out;
    bp.raw = raw;
    bp.b1 = key->b1;
    for (int u = 0; u < BL_P1_MAX; ++u) bp.k1[u] = key->k1[u];
    bp.tile_ctr = reinterpret_cast<unsigned *>(scr + 32);
    bp.big_count = reinterpret_cast<unsigned long long *>(scr + 8);
    bp.big_next = reinterpret_cast<unsigned long long *>(scr + 16);
    bp.pool_next = reinterpret_cast<unsigned long long *>(scr + 24);
    bp.big_str = reinterpret_cast<int64_t *>(scr + bs.big_str);
    bp.big_pool = reinterpret_cast<int64_t *>(scr + bs.big_pool);
    bp.big_seg = reinterpret_cast<int32_t *>(scr + bs.big_seg);
    bp.pool = scr + bs.pool;
    bp.big_cap = bs.big_cap;
    bp.pool_cap = bs.pool_cap;
    bp.status = d_status;
    // the chunk kernel runs only when the covered bytes can hold a string it
    // takes (otherwise its list gets no capacity, so that a batch larger than
    // its scratch claims reports PMP_ESCRATCH)
    const uint64_t chunk_bytes = (uint64_t)M * (N / 8);
    const bool big_needed = lo >= (BIG_CHUNKS - 1) * chunk_bytes;
    if (!big_needed) bp.big_cap = 0;

    cudaError_t e = cudaMemsetAsync(d_scratch, 0, 64, stream);
    if (e != cudaSuccess) return cuda_fail(e);
    if (g_batch_sched == PMP_BATCH_SORTED) {
        // one block per range at most, one wave of resident blocks
        if (g_batch_range == 1024)
            launch_range<N, RangeWide>(bp, n, dev->sms * dev->range_blocks_per_sm[N == 64][1], stream);
        else
            launch_range<N, RangeNarrow>(bp, n, dev->sms * dev->range_blocks_per_sm[N == 64][0], stream);
    } else {
        // enough warps that each takes at least one tile, at most the resident ones
        constexpr int64_t per_block = (int64_t)BL_T * BL_WARPS;  // strings per round of a block
        const int64_t blocks = (n + per_block - 1) / per_block;
        const int64_t cap = (int64_t)dev->sms * dev->lane_blocks_per_sm[N == 64][g_batch_p1 == 8];
        const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
        if (g_batch_p1 == 8)
            k_batch_lane<N, 8><<<grid, BL_THREADS, 0, stream>>>(bp);
        else
            k_batch_lane<N, 6><<<grid, BL_THREADS, 0, stream>>>(bp);
    }
    e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e);
    if (big_needed) {
        const int s3 = g_chunk_stages[N == 64] == 3;
        const unsigned cgrid = (unsigned)dev->sms * dev->chunk_blocks_per_sm[N == 64][s3];
        e = s3 ? launch_chunk_kernel<N, 3>(bp, cgrid, stream) : launch_chunk_kernel<N, 2>(bp, cgrid, stream);
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return PMP_OK;
}

template <int N>
int hash_fixed(const pmp_key *key, const uint8_t *d_keys, int64_t n, uint32_t len, uint64_t stride, void *d_out,
               cudaStream_t stream) {
    if (!key || key->width != N || n < 0 || (n > 0 && (!d_keys || !d_out))) return PMP_EINVAL;
    if ((uint64_t)len >= (uint64_t)M * (N / 8) || stride < len) return PMP_EINVAL;
    if ((stride & 7) || (reinterpret_cast<uintptr_t>(d_keys) & 7)) return PMP_EALIGN;
    if (n == 0) return PMP_OK;
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    FixedParams fp;
    memset(&fp, 0, sizeof fp);
    for (int u = 0; u < M; ++u) fp.k1[u] = key->k1[u];
    fp.b1 = key->b1;
    fp.base = d_keys;
    fp.stride = stride;
    fp.n = n;
    fp.len = len;
    fp.out = d_out;
    if (len <= 8) {
        // one unit: full key words rebuilt from their split halves
        auto word = [&](int u, int h) -> uint64_t {
            const uint4 k = key->k1[u];
            if (N == 32) return h ? ((uint64_t)k.z | ((uint64_t)k.w << 16)) : ((uint64_t)k.x | ((uint64_t)k.y << 16));
            return (uint64_t)k.x | ((uint64_t)k.y << 25) | ((uint64_t)k.z << 50);
        };
        fp.a0 = word(0, 0);
        fp.a1 = N == 32 ? word(0, 1) : 0;
        const uint64_t padw = len == 8 ? word(1, 0) : 0;  // the key word of the pad word 1
        fp.c_lo = key->b1 + padw;
        fp.c_hi = fp.c_lo < padw ? 1 : 0;
        const int64_t per_block = 256 * 2;  // two keys per thread
        const int64_t blocks = (n + per_block - 1) / per_block, cap = (int64_t)dev->sms * dev->fixed_blocks_per_sm[N == 64][2];
        k_fixed_one<N><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, stream>>>(fp);
        return cuda_fail(cudaGetLastError());
    }
    if (len <= 8 * FIXED_FEW_MAX) {
        // 2..9 units: full key words of the unit positions, and the pad's
        auto word = [&](int u, int h) -> uint64_t {
            const uint4 k = key->k1[u];
            if (N == 32) return h ? ((uint64_t)k.z | ((uint64_t)k.w << 16)) : ((uint64_t)k.x | ((uint64_t)k.y << 16));
            return (uint64_t)k.x | ((uint64_t)k.y << 25) | ((uint64_t)k.z << 50);
        };
        for (int u = 0; u < FIXED_FEW_MAX; ++u) fp.kw[u] = N == 32 ? word(u, 0) | (word(u, 1) << 32) : word(u, 0);
        const uint64_t padw = (len & 7) ? 0 : word((int)(len >> 3), 0);  // the key word of the pad word 1
        fp.pad_kw = padw;
        fp.c_lo = key->b1 + padw;
        fp.c_hi = fp.c_lo < padw ? 1 : 0;
        const int tier = len <= 16 ? 3 : len <= 40 ? 1 : 4;  // 2, 5 or 9 units
        // 16-byte loads only at strides of 64 bytes and more (measured: they
        // speed up 64-byte keys and slow down 16-, 32- and 48-byte ones)
        const bool v16 = !((reinterpret_cast<uintptr_t>(d_keys) & 15) || (stride & 63));
        const bool one_key = v16 && tier == 4;  // that instance takes one key per thread
        const int per_sm = dev->fixed_blocks_per_sm[N == 64][one_key ? 5 : tier];
        const int64_t per_block = 256 * (one_key ? 1 : 2);
        const int64_t blocks = (n + per_block - 1) / per_block, cap = (int64_t)dev->sms * per_sm;
        const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
        if (tier == 3)
            v16 ? k_fixed_few<N, 2, true><<<grid, 256, 0, stream>>>(fp) : k_fixed_few<N, 2, false><<<grid, 256, 0, stream>>>(fp);
        else if (tier == 1)
            v16 ? k_fixed_few<N, 5, true><<<grid, 256, 0, stream>>>(fp) : k_fixed_few<N, 5, false><<<grid, 256, 0, stream>>>(fp);
        else
            v16 ? k_fixed_few<N, FIXED_FEW_MAX, true><<<grid, 256, 0, stream>>>(fp)
                : k_fixed_few<N, FIXED_FEW_MAX, false><<<grid, 256, 0, stream>>>(fp);
        return cuda_fail(cudaGetLastError());
    }
    // one wave of resident blocks, one key per thread
    const int64_t blocks = (n + 255) / 256, cap = (int64_t)dev->sms * dev->fixed_blocks_per_sm[N == 64][0];
    k_fixed<N><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, stream>>>(fp);
    return cuda_fail(cudaGetLastError());
}

template <int N>
int hash_plain(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets, int64_t n,
               void *d_out, cudaStream_t stream) {
    if (!key || key->width != N || n < 0 || (n > 0 && (!d_offsets || !d_out || !d_base)))
        return PMP_EINVAL;
    if (reinterpret_cast<uintptr_t>(d_base) & 7) return PMP_EALIGN;
    typedef typename Fam<N>::word word;
    for (int64_t i = 0; i < n; ++i) {
        k_plain<N><<<1, 32, 0, stream>>>(d_base, d_offsets, i,
                                         static_cast<const word *>(key->d_words), d_out);
        cudaError_t e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
    }
    return PMP_OK;
}

// Fixed scratch of pmp_hash64_noalloc: one array per device, compiled into
// the library. Host code only sees a stand-in symbol; the device address is
// looked up once per device with cudaGetSymbolAddress.
constexpr size_t NOALLOC_SCRATCH_BYTES = 1u << 20;
__device__ __align__(256) uint8_t g_noalloc_scratch[NOALLOC_SCRATCH_BYTES];
void *g_noalloc_ptr[MAX_DEVICES];
std::mutex g_noalloc_mu;

}  // namespace

struct pmp_graph {
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

// Capture one call on a private stream into an executable graph. The
// per-device set-up runs before the capture.
template <class F>
int capture(F call, pmp_graph **out) {
    if (!out) return PMP_EINVAL;
    *out = nullptr;
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    cudaStream_t s;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return cuda_fail(cudaGetLastError());
    cudaGraph_t g = nullptr;
    cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
        rc = call(s);
        e = cudaStreamEndCapture(s, &g);
    }
    cudaStreamDestroy(s);
    if (e != cudaSuccess || rc) {
        if (g) cudaGraphDestroy(g);
        return rc ? rc : cuda_fail(e);
    }
    cudaGraphExec_t x = nullptr;
    e = cudaGraphInstantiate(&x, g, 0);
    if (e != cudaSuccess) {
        cudaGraphDestroy(g);
        return cuda_fail(e);
    }
    pmp_graph *gr = new pmp_graph;
    gr->graph = g;
    gr->exec = x;
    *out = gr;
    return PMP_OK;
}

}  // namespace

extern "C" {

int pmp_key_create(uint64_t seed, int width, pmp_key **out) {
    if (!out || (width != 32 && width != 64)) return PMP_EINVAL;
    *out = nullptr;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    void *d = nullptr;
    e = cudaMalloc(&d, key_bytes(width));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        return PMP_ENOMEM;
    }
    if (width == 32)
        k_keygen<32><<<1, 32>>>(seed, static_cast<uint32_t *>(d));
    else
        k_keygen<64><<<1, 32>>>(seed, static_cast<uint64_t *>(d));
    e = cudaGetLastError();
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e != cudaSuccess) {
        cudaFree(d);
        return cuda_fail(e);
    }
    pmp_key *k = new pmp_key;
    k->width = width;
    k->device = dev;
    k->d_words = d;
    // level-1 row (b_1, a_{1,1..m}) on the host, split as the kernels split it
    uint64_t row[KEY_ROW];
    if (width == 32) {
        uint32_t r32[KEY_ROW];
        e = cudaMemcpy(r32, d, sizeof r32, cudaMemcpyDeviceToHost);
        for (int i = 0; i < KEY_ROW; ++i) row[i] = r32[i];
    } else {
        e = cudaMemcpy(row, d, sizeof row, cudaMemcpyDeviceToHost);
    }
    if (e != cudaSuccess) {
        cudaFree(d);
        delete k;
        return cuda_fail(e);
    }
    k->b1 = row[0];
    for (int u = 0; u < (width == 32 ? M / 2 : M); ++u) {
        if (width == 32) {
            const uint64_t a0 = row[1 + 2 * u], a1 = row[2 + 2 * u];
            k->k1[u] = make_uint4((uint32_t)(a0 & 0xffffu), (uint32_t)(a0 >> 16), (uint32_t)(a1 & 0xffffu),
                                  (uint32_t)(a1 >> 16));
        } else {
            const uint64_t a = row[1 + u];
            k->k1[u] = make_uint4((uint32_t)(a & 0x1ffffffull), (uint32_t)((a >> 25) & 0x1ffffffull),
                                  (uint32_t)(a >> 50), 0u);
        }
    }
    *out = k;
    return PMP_OK;
}

int pmp_key_export(const pmp_key *key, void *host_dst, size_t cap_bytes) {
    if (!key || !host_dst || cap_bytes < key_bytes(key->width)) return PMP_EINVAL;
    return cuda_fail(cudaMemcpy(host_dst, key->d_words, key_bytes(key->width), cudaMemcpyDeviceToHost));
}

int pmp_key_width(const pmp_key *key) { return key ? key->width : 0; }

void pmp_key_destroy(pmp_key *key) {
    if (!key) return;
    cudaDeviceSynchronize();
    cudaFree(key->d_words);
    delete key;
}

size_t pmp_hash_scratch_bytes(int width, uint64_t len) {
    Plan p;
    if ((width != 32 && width != 64) || make_plan(width, len, p)) return 0;
    return p.scratch;
}

int pmp_hash32(const pmp_key *key, const void *d_buf, uint64_t len, uint32_t *d_out,
               void *d_scratch, size_t scratch_bytes, void *stream) {
    return hash_one<32>(key, d_buf, len, d_out, nullptr, d_scratch, scratch_bytes,
                        static_cast<cudaStream_t>(stream));
}

int pmp_hash64(const pmp_key *key, const void *d_buf, uint64_t len, uint64_t *d_out,
               void *d_scratch, size_t scratch_bytes, void *stream) {
    return hash_one<64>(key, d_buf, len, d_out, nullptr, d_scratch, scratch_bytes,
                        static_cast<cudaStream_t>(stream));
}

int pmp_hash_fixed32(const pmp_key *key, const uint8_t *d_keys, int64_t n, uint32_t len, uint64_t stride,
                     uint32_t *d_out, void *stream) {
    return hash_fixed<32>(key, d_keys, n, len, stride, d_out, static_cast<cudaStream_t>(stream));
}

int pmp_hash_fixed64(const pmp_key *key, const uint8_t *d_keys, int64_t n, uint32_t len, uint64_t stride,
                     uint64_t *d_out, void *stream) {
    return hash_fixed<64>(key, d_keys, n, len, stride, d_out, static_cast<cudaStream_t>(stream));
}

int pmp_count_collisions(int width, uint64_t seed0, uint64_t nkeys, const uint8_t *d_a, uint32_t len_a,
                         const uint8_t *d_b, uint32_t len_b, int t_bits, unsigned long long *d_count,
                         void *stream) {
    if ((width != 32 && width != 64) || !d_a || !d_b || !d_count || t_bits < 1 || t_bits > width)
        return PMP_EINVAL;
    const uint64_t W = (uint64_t)width / 8;
    if (len_a / W + 1 > (uint64_t)COLLIDE_MAX_WORDS || len_b / W + 1 > (uint64_t)COLLIDE_MAX_WORDS)
        return PMP_EINVAL;
    if ((reinterpret_cast<uintptr_t>(d_a) | reinterpret_cast<uintptr_t>(d_b)) & 7) return PMP_EALIGN;
    if (nkeys == 0) return PMP_OK;
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    const uint64_t blocks = (nkeys + 255) / 256, cap = (uint64_t)dev->sms * 8;
    const unsigned grid = (unsigned)(blocks < cap ? blocks : cap);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (width == 32)
        k_collide<32><<<grid, 256, 0, st>>>(seed0, nkeys, d_a, len_a, d_b, len_b, t_bits, d_count);
    else
        k_collide<64><<<grid, 256, 0, st>>>(seed0, nkeys, d_a, len_a, d_b, len_b, t_bits, d_count);
    return cuda_fail(cudaGetLastError());
}

static int toy_params(int n, int kappa, int m, int L, ToyParams *P) {
    if ((n != 8 && n != 16) || kappa < 0 || m < 2 || m > TOY_MAXM || L < 1 || L > TOY_MAXL) return PMP_EINVAL;
    if ((uint32_t)kappa >= (1u << n)) return PMP_EINVAL;  // p - kappa - 1 >= 1 key value
    *P = ToyParams{(uint32_t)n, 1u, (uint32_t)kappa, (uint32_t)m, (uint32_t)L};
    return PMP_OK;
}

int pmp_toy_regularity(int n, int kappa, int m, int L, uint64_t seed0, uint32_t nkeys, const uint8_t *d_str,
                       uint32_t len, uint32_t comp0, uint32_t ncomp, uint32_t *d_counts, uint32_t *d_raw,
                       void *stream) {
    ToyParams P;
    int rc = toy_params(n, kappa, m, L, &P);
    if (rc) return rc;
    const uint32_t W = (uint32_t)n / 8, N0 = len / W + 1;
    if (!d_counts || (len && !d_str) || N0 > (uint32_t)TOY_MAXW) return PMP_EINVAL;
    if ((uint64_t)comp0 + ncomp > len / W) return PMP_EINVAL;  // whole string words only
    uint32_t lv = 0, N = N0;
    do {
        N = (N + (uint32_t)m - 1) / (uint32_t)m;
        ++lv;
    } while (N > 1);
    if (lv > (uint32_t)L) return PMP_ETOOLONG;
    if (nkeys == 0 || ncomp == 0) return PMP_OK;
    if ((uint64_t)nkeys * ncomp > 0x7fffffffull) return PMP_EINVAL;
    k_toy_regular<<<nkeys * ncomp, TOY_THREADS, 0, static_cast<cudaStream_t>(stream)>>>(P, seed0, ncomp, comp0, d_str,
                                                                                        len, d_counts, d_raw);
    return cuda_fail(cudaGetLastError());
}

int pmp_toy_delta_hist(int n, int kappa, int m, const uint32_t *s, const uint32_t *t, unsigned long long *d_hist,
                       void *stream) {
    ToyParams P;
    int rc = toy_params(n, kappa, m, 1, &P);
    if (rc) return rc;
    if (!s || !t || !d_hist) return PMP_EINVAL;
    const uint32_t p = (1u << n) + 1u, R = p - (uint32_t)kappa - 1;
    ToyDelta D;
    int first = -1;
    for (int i = 0; i < m; ++i) {
        if (s[i] >= p || t[i] >= p) return PMP_EINVAL;
        D.d[i] = (s[i] + p - t[i]) % p;
        if (D.d[i] && first < 0) first = i;
    }
    if (first < 0) return PMP_EINVAL;  // s == t
    const uint32_t d0 = D.d[0];        // swapping two components permutes the key set: same histogram
    D.d[0] = D.d[first];
    D.d[first] = d0;
    uint64_t outer = 1;
    for (int i = 1; i < m; ++i) {
        outer *= R;
        if (outer * R > (1ull << 40)) return PMP_EINVAL;  // at most 2^40 keys
    }
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    if (cudaMemsetAsync(d_hist, 0, (size_t)p * sizeof(unsigned long long), st) != cudaSuccess) return PMP_ECUDA;
    DeviceInfo *dev;
    rc = device_info(&dev);
    if (rc) return rc;
    const uint64_t warps = TOY_THREADS / 32, blocks = (outer + warps - 1) / warps, cap = (uint64_t)dev->sms * 8;
    k_toy_delta<<<(unsigned)(blocks < cap ? blocks : cap), TOY_THREADS, 0, st>>>(P, D, outer, d_hist);
    return cuda_fail(cudaGetLastError());
}

size_t pmp_batch_scratch_bytes(int width, int64_t n, uint64_t data_bytes) {
    if (width != 32 && width != 64) return 0;
    if (n < 0) return 0;
    return batch_scratch(width, data_bytes).total;
}

int pmp_hash_batch32(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                     int64_t n, uint32_t *d_out, void *d_scratch, size_t scratch_bytes,
                     void *stream) {
    return hash_batch<32>(key, d_base, d_offsets, n, d_out, 0, d_scratch, scratch_bytes,
                          static_cast<cudaStream_t>(stream));
}

int pmp_hash_batch64(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                     int64_t n, uint64_t *d_out, void *d_scratch, size_t scratch_bytes,
                     void *stream) {
    return hash_batch<64>(key, d_base, d_offsets, n, d_out, 0, d_scratch, scratch_bytes,
                          static_cast<cudaStream_t>(stream));
}

int pmp_hash_batch_status(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets, int64_t n,
                          void *d_out, int *d_status, void *d_scratch, size_t scratch_bytes, void *stream) {
    if (!key || !d_status) return PMP_EINVAL;
    if (key->width == 32)
        return hash_batch<32>(key, d_base, d_offsets, n, d_out, 0, d_scratch, scratch_bytes,
                              static_cast<cudaStream_t>(stream), d_status);
    return hash_batch<64>(key, d_base, d_offsets, n, d_out, 0, d_scratch, scratch_bytes,
                          static_cast<cudaStream_t>(stream), d_status);
}

int pmp_hash_batch_raw(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                       int64_t n, uint64_t *d_raw, void *d_scratch, size_t scratch_bytes,
                       void *stream) {
    if (!key) return PMP_EINVAL;
    if (key->width == 32)
        return hash_batch<32>(key, d_base, d_offsets, n, d_raw, 1, d_scratch, scratch_bytes,
                              static_cast<cudaStream_t>(stream));
    return hash_batch<64>(key, d_base, d_offsets, n, d_raw, 1, d_scratch, scratch_bytes,
                          static_cast<cudaStream_t>(stream));
}

int pmp_hash_batch32_plain(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                           int64_t n, uint32_t *d_out, void *stream) {
    return hash_plain<32>(key, d_base, d_offsets, n, d_out, static_cast<cudaStream_t>(stream));
}

int pmp_hash_batch64_plain(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                           int64_t n, uint64_t *d_out, void *stream) {
    return hash_plain<64>(key, d_base, d_offsets, n, d_out, static_cast<cudaStream_t>(stream));
}

int pmp_debug_reduce(int width, const uint64_t *d_S, int64_t n, uint64_t *d_z, void *stream) {
    if ((width != 32 && width != 64) || n < 0 || (n > 0 && (!d_S || !d_z))) return PMP_EINVAL;
    if (n == 0) return PMP_OK;
    const unsigned grid = (unsigned)((n + 255) / 256);
    cudaStream_t s = static_cast<cudaStream_t>(stream);
    if (width == 32)
        k_debug_reduce<32><<<grid, 256, 0, s>>>(d_S, n, d_z);
    else
        k_debug_reduce<64><<<grid, 256, 0, s>>>(d_S, n, d_z);
    return cuda_fail(cudaGetLastError());
}

static int check_grid(unsigned *grid) {
    DeviceInfo *dev;
    const int rc = device_info(&dev);
    if (rc) return rc;
    *grid = (unsigned)dev->sms * 8;
    return PMP_OK;
}

int pmp_check_alg2_32(unsigned long long *d_bad, void *stream) {
    if (!d_bad) return PMP_EINVAL;
    unsigned grid;
    int rc = check_grid(&grid);
    if (rc) return rc;
    k_check_alg2_32<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(d_bad);
    return cuda_fail(cudaGetLastError());
}

int pmp_check_reduce32(const uint32_t *r1, const uint32_t *r2, int npairs, unsigned long long *d_bad,
                       void *stream) {
    if (!d_bad || !r1 || !r2 || npairs < 1 || npairs > CHECK_MAX_PAIRS) return PMP_EINVAL;
    CheckPairs P;
    P.n = npairs;
    for (int j = 0; j < npairs; ++j) {
        if (r2[j] > (uint32_t)M) return PMP_EINVAL;  // three-word sums of Sec. 6.2: w2 <= m
        P.r1[j] = r1[j];
        P.r2[j] = r2[j];
    }
    unsigned grid;
    int rc = check_grid(&grid);
    if (rc) return rc;
    k_check_reduce32<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(P, d_bad);
    return cuda_fail(cudaGetLastError());
}

int pmp_check_mix32(uint32_t a_inv, unsigned long long *d_bad, void *stream) {
    if (!d_bad) return PMP_EINVAL;
    unsigned grid;
    int rc = check_grid(&grid);
    if (rc) return rc;
    k_check_mix32<<<grid, 256, 0, static_cast<cudaStream_t>(stream)>>>(a_inv, d_bad);
    return cuda_fail(cudaGetLastError());
}

int pmp_debug_wait_timeout(int *d_result, void *stream) {
    if (!d_result) return PMP_EINVAL;
    k_wait_probe<<<1, 32, 0, static_cast<cudaStream_t>(stream)>>>(d_result);
    return cuda_fail(cudaGetLastError());
}

int pmp_device_status(int *out) {
    if (!out) return PMP_EINVAL;
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) return cuda_fail(e);
    int v = 0;
    e = cudaMemcpyFromSymbol(&v, g_device_status, sizeof v);
    if (e != cudaSuccess) return cuda_fail(e);
    const int zero = 0;
    e = cudaMemcpyToSymbol(g_device_status, &zero, sizeof zero);
    if (e != cudaSuccess) return cuda_fail(e);
    *out = v;
    return PMP_OK;
}

uint64_t pmp_hash_noalloc_max_len(void) {
    // the scratch need grows with len: largest len whose plan fits (bisection)
    uint64_t lo = 0, hi = 1ull << 60;
    while (lo < hi) {
        const uint64_t mid = lo + (hi - lo + 1) / 2;
        Plan p;
        if (make_plan(64, mid, p) == PMP_OK && p.scratch <= NOALLOC_SCRATCH_BYTES)
            lo = mid;
        else
            hi = mid - 1;
    }
    return lo;
}

int pmp_hash64_noalloc(const pmp_key *key, const void *d_buf, uint64_t len, uint64_t *d_out,
                       void *stream) {
    Plan plan;
    const int rc = make_plan(64, len, plan);
    if (rc) return rc;
    if (plan.scratch > NOALLOC_SCRATCH_BYTES) return PMP_ESCRATCH;
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e);
    if (dev < 0 || dev >= MAX_DEVICES) return PMP_EINVAL;
    void *scratch = nullptr;
    {
        std::lock_guard<std::mutex> lk(g_noalloc_mu);
        if (!g_noalloc_ptr[dev]) {
            e = cudaGetSymbolAddress(&g_noalloc_ptr[dev], g_noalloc_scratch);
            if (e != cudaSuccess) {
                g_noalloc_ptr[dev] = nullptr;
                return cuda_fail(e);
            }
        }
        scratch = g_noalloc_ptr[dev];
    }
    return hash_one<64>(key, d_buf, len, d_out, nullptr, scratch, NOALLOC_SCRATCH_BYTES,
                        static_cast<cudaStream_t>(stream));
}

int pmp_graph_hash(const pmp_key *key, const void *d_buf, uint64_t len, void *d_out, void *d_scratch,
                   size_t scratch_bytes, pmp_graph **out) {
    if (!key) return PMP_EINVAL;
    return capture(
        [&](cudaStream_t s) {
            return key->width == 32
                       ? hash_one<32>(key, d_buf, len, d_out, nullptr, d_scratch, scratch_bytes, s)
                       : hash_one<64>(key, d_buf, len, d_out, nullptr, d_scratch, scratch_bytes, s);
        },
        out);
}

int pmp_graph_batch(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets, int64_t n,
                    void *d_out, void *d_scratch, size_t scratch_bytes, pmp_graph **out) {
    if (!key) return PMP_EINVAL;
    return capture(
        [&](cudaStream_t s) {
            return key->width == 32
                       ? hash_batch<32>(key, d_base, d_offsets, n, d_out, 0, d_scratch, scratch_bytes, s)
                       : hash_batch<64>(key, d_base, d_offsets, n, d_out, 0, d_scratch, scratch_bytes, s);
        },
        out);
}

int pmp_graph_launch(pmp_graph *g, void *stream) {
    if (!g) return PMP_EINVAL;
    return cuda_fail(cudaGraphLaunch(g->exec, static_cast<cudaStream_t>(stream)));
}

void pmp_graph_destroy(pmp_graph *g) {
    if (!g) return;
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    delete g;
}

// ---------------------------------------------------------------------------
// Streaming (incremental) hashing of one string delivered in pieces.
// ---------------------------------------------------------------------------
}  // extern "C"

struct pmp_stream {
    const pmp_key *key = nullptr;
    int width = 0;
    StreamState *d_state = nullptr;
    Val *d_vals[2] = {nullptr, nullptr};  // level values of one segment (ping-pong)
    uint64_t total = 0;                   // bytes absorbed
    uint32_t carry_len = 0;               // bytes in the incomplete level-1 chunk
    int cb = 0;                           // carry buffer holding them
    uint64_t count[LMAX + 2] = {0};       // values received by each level (levels >= 2)
    uint32_t cur = 0;                     // bit L: current partial-sum buffer of level L
    Val *d_l2 = nullptr;                  // level-2 values not yet folded into level 3
    uint64_t l2_pending = 0;              // how many
    uint64_t tiles_claimed = 0;           // the tree kernel's work counter in the state (never reset)
};

namespace {

// Level-1 chunks hashed per launch of the update kernels (the value buffers
// hold one such segment).
constexpr uint64_t STREAM_SEG_CHUNKS = 1u << 19;
// segments of at least this many whole chunks at a 16-byte aligned address
// go through the tree kernel (level-2 output mode when the segment starts a
// level-2 chunk, else level-1 output mode)
constexpr uint64_t STREAM_TREE_MIN = 4096;
// level-2 values that wait to be folded into levels 3 and up
constexpr uint64_t STREAM_L2_CAP = 1u << 19;

// The fold of the waiting level-2 values into level 3 and up: its launch
// shape and level bookkeeping (the host's counts and buffer selectors are
// advanced as if it had run).
struct FlushPlan {
    uint64_t n, c3, n3;
    unsigned grid;
    int src3;
    FoldRest fr;
};

int flush_plan(pmp_stream *s, const DeviceInfo *dev, FlushPlan &f) {
    f.n = s->l2_pending;
    f.c3 = s->count[3];
    f.n3 = (f.c3 + f.n) / M - f.c3 / M;
    const uint64_t chunks = (f.c3 + f.n - 1) / M - f.c3 / M + 1;
    const uint64_t blocks = (chunks + 7) / 8, cap = (uint64_t)dev->sms * 16;
    f.grid = (unsigned)(blocks < cap ? blocks : cap);
    f.src3 = (int)((s->cur >> 3) & 1);
    s->cur ^= 1u << 3;
    s->count[3] += f.n;
    memset(&f.fr, 0, sizeof f.fr);
    f.fr.cur = s->cur;
    uint64_t nl = f.n3;
    for (int L = 4; nl > 0 && L <= LMAX; ++L) {
        f.fr.c_old[L] = s->count[L];
        const uint64_t next = (s->count[L] + nl) / M - s->count[L] / M;
        s->count[L] += nl;
        s->cur ^= 1u << L;
        nl = next;
    }
    s->l2_pending = 0;
    return PMP_OK;
}

// Levels 3 and up of the level-2 values that waited (the level-2 mode of the
// tree kernel): one warp per touched chunk of level 3, levels 4 and up by
// the fold's last block.
template <int N>
int stream_flush(pmp_stream *s, cudaStream_t stream) {
    typedef typename Fam<N>::word word;
    if (s->l2_pending == 0) return PMP_OK;
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    FlushPlan f;
    flush_plan(s, dev, f);
    k_stream_fold<N><<<f.grid, 256, 0, stream>>>(s->d_state, static_cast<const word *>(s->key->d_words), 3,
                                                  s->d_l2, f.c3, f.n, f.src3, s->d_vals[1], f.n3, f.fr,
                                                  s->d_vals[0]);
    return cuda_fail(cudaGetLastError());
}

// A launch as a programmatic dependent of the kernel before it on the stream:
// its blocks may be scheduled once that kernel has triggered (a level-2 mode
// tree launch does after its last tile claims) and load the key rows, then
// wait (griddepcontrol.wait) for its completion; after a copy or a kernel
// that does not trigger, it starts as any launch does.
template <typename... KArgs, typename... Args>
cudaError_t launch_dependent(void (*kern)(KArgs...), unsigned grid, unsigned block, cudaStream_t stream,
                             Args &&...args) {
    cudaLaunchConfig_t cfg = {};
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(block);
    cfg.dynamicSmemBytes = 0;
    cfg.stream = stream;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, kern, std::forward<Args>(args)...);
}

// The result: with level-2 values waiting, their fold and the final chunk in
// one launch (k_stream_finish); otherwise the final chunk alone. Either is a
// programmatic dependent of the launch before it.
template <int N>
int stream_result(pmp_stream *s, void *d_out, uint64_t *d_raw, cudaStream_t stream) {
    typedef typename Fam<N>::word word;
    const word *key = static_cast<const word *>(s->key->d_words);
    StreamCounts counts;
    memset(&counts, 0, sizeof counts);
    if (s->l2_pending == 0) {
        for (int j = 0; j < LMAX + 2; ++j) counts.total[j] = s->count[j];
        return cuda_fail(launch_dependent(k_stream_final<N>, 1, 32, stream, s->d_state, key, s->cb, s->carry_len,
                                          s->cur, counts, d_out, d_raw));
    }
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    FlushPlan f;
    flush_plan(s, dev, f);
    for (int j = 0; j < LMAX + 2; ++j) counts.total[j] = s->count[j];
    return cuda_fail(launch_dependent(k_stream_finish<N>, f.grid, 256, stream, s->d_state, key, s->d_l2, f.c3, f.n,
                                      f.src3, s->d_vals[1], f.n3, f.fr, s->d_vals[0], s->cb, s->carry_len, s->cur,
                                      counts, d_out, d_raw));
}

template <int N>
int stream_update(pmp_stream *s, const uint8_t *piece, uint64_t len, cudaStream_t stream) {
    typedef typename Fam<N>::word word;
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;
    if (len == 0) return PMP_OK;
    Plan plan;
    if (s->total + len < s->total || make_plan(N, s->total + len, plan)) return PMP_ETOOLONG;
    DeviceInfo *dev;
    int rc = device_info(&dev);
    if (rc) return rc;
    const word *key = static_cast<const word *>(s->key->d_words);
    uint8_t *carry = s->d_state->carry[s->cb];
    cudaError_t e;
    if (s->carry_len + len < CB) {  // the chunk is still incomplete
        e = cudaMemcpyAsync(carry + s->carry_len, piece, len, cudaMemcpyDeviceToDevice, stream);
        if (e != cudaSuccess) return cuda_fail(e);
        s->carry_len += (uint32_t)len;
        s->total += len;
        return PMP_OK;
    }
    const uint64_t head = s->carry_len ? CB - s->carry_len : 0;  // bytes that complete the carried chunk
    const uint8_t *body = piece + head;
    const uint64_t nbody = (len - head) / CB, rem = (len - head) % CB;
    uint8_t *tail_dst = s->d_state->carry[s->cb ^ 1];
    uint64_t done = 0;
    bool first = true;
    const unsigned cap = (unsigned)dev->sms * 16;
    while ((first && s->carry_len) || done < nbody) {
        const int use_carry = first && s->carry_len ? 1 : 0;
        const uint64_t room = (uint64_t)g_stream_segment - (uint64_t)use_carry;
        const uint64_t nb = nbody - done < room ? nbody - done : room;
        const bool last = done + nb == nbody;
        const uint64_t n = (uint64_t)use_carry + nb;
        const uint8_t *seg = body + done * CB;
        const bool tree_ok = nb >= STREAM_TREE_MIN && (reinterpret_cast<uintptr_t>(seg) & 15) == 0;
        if (tree_ok && !use_carry && s->count[2] % M == 0) {
            // the segment starts a level-2 chunk: the tree kernel's combiner
            // forms the level-2 values (level-1 values stay on chip); levels 3
            // and up wait in d_l2
            if (s->l2_pending + nb / M + 1 > STREAM_L2_CAP) {
                rc = stream_flush<N>(s, stream);
                if (rc) return rc;
            }
            const int src2 = (int)((s->cur >> 2) & 1);
            TreeParams tp;
            memset(&tp, 0, sizeof tp);
            tp.buf = seg;
            tp.len = nb * CB;
            tp.F = nb;
            tp.c[1] = nb;
            tp.c[2] = (nb + M - 1) / M;
            tp.levels = 2;
            tp.key = key;
            tp.use_tma = 1;
            tp.l2_out = s->d_l2 + s->l2_pending;
            tp.l2_part = &s->d_state->sum[src2 ^ 1][2];
            tp.l2_first = s->count[2] == 0 ? &s->d_state->first[2] : nullptr;
            tp.tile_ctr = &s->d_state->tile_ctr;
            CUtensorMap tmap;
            memset(&tmap, 0, sizeof tmap);
            rc = encode_chunk_map<N>(seg, nb, tmap);
            if (rc) return rc;
            // the counter runs on across launches: each producer claims its
            // tiles and one past the end, then triggers, so that the next
            // level-2 launch (a programmatic dependent) claims only after
            // every claim of this one
            tp.tile_base = s->tiles_claimed;
            s->tiles_claimed += tp.c[2] + tree_grid<N>(dev, tp.c[2]);
            tp.trigger = 1;
            rc = launch_tree<N>(dev, tmap, tp, tp.c[2], stream, true);
            if (rc) return rc;
            if (last && rem) {
                e = cudaMemcpyAsync(tail_dst, body + nbody * CB, rem, cudaMemcpyDeviceToDevice, stream);
                if (e != cudaSuccess) return cuda_fail(e);
            }
            s->cur ^= 1u << 2;
            s->count[2] += nb;
            s->l2_pending += nb / M;
            done += nb;
            first = false;
            continue;
        }
        // any other update folds into level 3 itself: the waiting values first
        rc = stream_flush<N>(s, stream);
        if (rc) return rc;
        if (tree_ok) {
            // the segment's whole chunks through the tree kernel's TMA pipeline
            // (level-1 output mode); the carried chunk and the remaining bytes
            // by the small kernel and a copy
            if (use_carry) {
                k_stream_l1<N><<<1, 256, 0, stream>>>(key, carry, s->carry_len, piece, seg, 0, seg, 0u,
                                                      tail_dst, s->d_vals[0]);
                e = cudaGetLastError();
                if (e != cudaSuccess) return cuda_fail(e);
            }
            TreeParams tp;
            memset(&tp, 0, sizeof tp);
            tp.buf = seg;
            tp.len = nb * CB;
            tp.F = nb;
            tp.c[1] = nb;
            tp.c[2] = (nb + M - 1) / M;
            tp.levels = 2;
            tp.key = key;
            tp.use_tma = 1;
            tp.l1_out = s->d_vals[0] + use_carry;
            tp.tile_ctr = &s->d_state->tile_ctr;
            CUtensorMap tmap;
            memset(&tmap, 0, sizeof tmap);
            rc = encode_chunk_map<N>(seg, nb, tmap);
            if (rc) return rc;
            // the counter runs on across launches: each producer claims its
            // tiles and one past the end
            tp.tile_base = s->tiles_claimed;
            s->tiles_claimed += tp.c[2] + tree_grid<N>(dev, tp.c[2]);
            rc = launch_tree<N>(dev, tmap, tp, tp.c[2], stream);
            if (rc) return rc;
            if (last && rem) {
                e = cudaMemcpyAsync(tail_dst, body + nbody * CB, rem, cudaMemcpyDeviceToDevice, stream);
                if (e != cudaSuccess) return cuda_fail(e);
            }
        } else {
            // 8 warps of 4 chunks per block; at most one wave of resident blocks
            // (the launch bounds guarantee 4 or 5 per SM), each warp looping
            const uint64_t l1_blocks = (n + 31) / 32;
            const unsigned l1_cap = (unsigned)dev->sms * (N == 64 ? 4 : 5);
            k_stream_l1<N><<<(unsigned)(l1_blocks < l1_cap ? l1_blocks : l1_cap), 256, 0, stream>>>(
                key, carry, use_carry ? s->carry_len : 0u, piece, seg, nb, body + nbody * CB,
                last ? (uint32_t)rem : 0u, tail_dst, s->d_vals[0]);
            e = cudaGetLastError();
            if (e != cudaSuccess) return cuda_fail(e);
        }
        // level 2: one warp per touched chunk
        const uint64_t c2 = s->count[2];
        const uint64_t n2 = (c2 + n) / M - c2 / M;
        const uint64_t chunks = (c2 + n - 1) / M - c2 / M + 1;
        const uint64_t blocks = (chunks + 7) / 8;
        const int src2 = (int)((s->cur >> 2) & 1);
        s->cur ^= 1u << 2;
        s->count[2] += n;
        // levels 3 and up (the fold's last block): the values each level held
        // before and its partial sum buffer
        FoldRest fr;
        memset(&fr, 0, sizeof fr);
        fr.cur = s->cur;
        uint64_t nl = n2;
        for (int L = 3; nl > 0 && L <= LMAX; ++L) {
            fr.c_old[L] = s->count[L];
            const uint64_t next = (s->count[L] + nl) / M - s->count[L] / M;
            s->count[L] += nl;
            s->cur ^= 1u << L;
            nl = next;
        }
        k_stream_fold<N><<<(unsigned)(blocks < cap ? blocks : cap), 256, 0, stream>>>(
            s->d_state, key, 2, s->d_vals[0], c2, n, src2, s->d_vals[1], n2, fr, s->d_vals[0]);
        e = cudaGetLastError();
        if (e != cudaSuccess) return cuda_fail(e);
        done += nb;
        first = false;
    }
    s->cb ^= 1;  // the last segment copied the remaining bytes to the other buffer
    s->carry_len = (uint32_t)rem;
    s->total += len;
    return PMP_OK;
}

}  // namespace

extern "C" {

int pmp_stream_create(const pmp_key *key, pmp_stream **out) {
    if (!out || !key) return PMP_EINVAL;
    *out = nullptr;
    pmp_stream *s = new pmp_stream;
    s->key = key;
    s->width = key->width;
    cudaError_t e = cudaMalloc(&s->d_state, sizeof(StreamState));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_vals[0], sizeof(Val) * STREAM_SEG_CHUNKS);
    if (e == cudaSuccess) e = cudaMalloc(&s->d_vals[1], sizeof(Val) * (STREAM_SEG_CHUNKS / M + 2));
    if (e == cudaSuccess) e = cudaMalloc(&s->d_l2, sizeof(Val) * STREAM_L2_CAP);
    if (e == cudaSuccess) e = cudaMemset(s->d_state, 0, sizeof(StreamState));
    if (e != cudaSuccess) {
        (void)cudaGetLastError();
        pmp_stream_destroy(s);
        return PMP_ENOMEM;
    }
    *out = s;
    return PMP_OK;
}

int pmp_stream_update(pmp_stream *s, const void *d_piece, uint64_t len, void *stream) {
    if (!s || (len && !d_piece)) return PMP_EINVAL;
    const uint8_t *p = static_cast<const uint8_t *>(d_piece);
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return s->width == 32 ? stream_update<32>(s, p, len, st) : stream_update<64>(s, p, len, st);
}

int pmp_stream_final(pmp_stream *s, void *d_out, uint64_t *d_raw, void *stream) {
    if (!s || !d_out) return PMP_EINVAL;
    cudaStream_t st = static_cast<cudaStream_t>(stream);
    return s->width == 32 ? stream_result<32>(s, d_out, d_raw, st) : stream_result<64>(s, d_out, d_raw, st);
}

int pmp_stream_reset(pmp_stream *s, void *stream) {
    if (!s) return PMP_EINVAL;
    cudaError_t e = cudaMemsetAsync(s->d_state, 0, sizeof(StreamState), static_cast<cudaStream_t>(stream));
    if (e != cudaSuccess) return cuda_fail(e);
    s->total = 0;
    s->carry_len = 0;
    s->cb = 0;
    s->cur = 0;
    s->l2_pending = 0;
    s->tiles_claimed = 0;  // the state's counter is zeroed with it
    for (int j = 0; j < LMAX + 2; ++j) s->count[j] = 0;
    return PMP_OK;
}

uint64_t pmp_stream_length(const pmp_stream *s) { return s ? s->total : 0; }

void pmp_stream_destroy(pmp_stream *s) {
    if (!s) return;
    cudaDeviceSynchronize();
    cudaFree(s->d_state);
    cudaFree(s->d_vals[0]);
    cudaFree(s->d_vals[1]);
    cudaFree(s->d_l2);
    delete s;
}

int pmp_tune_set(int knob, int value) {
    switch (knob) {
        case PMP_KNOB_TREE_STAGES_32:
        case PMP_KNOB_TREE_STAGES_64:
            if (stage_index(value) < 0) return PMP_EINVAL;
            g_tree_stages[knob == PMP_KNOB_TREE_STAGES_64] = value;
            return PMP_OK;
        case PMP_KNOB_BATCH_P1:
            if (value != 6 && value != 8) return PMP_EINVAL;
            g_batch_p1 = value;
            return PMP_OK;
        case PMP_KNOB_BATCH_SCHED:
            if (value != PMP_BATCH_SORTED && value != PMP_BATCH_TILES) return PMP_EINVAL;
            g_batch_sched = value;
            return PMP_OK;
        case PMP_KNOB_BATCH_RANGE:
            if (value != 512 && value != 1024) return PMP_EINVAL;
            g_batch_range = value;
            return PMP_OK;
        case PMP_KNOB_CHUNK_STAGES_32:
        case PMP_KNOB_CHUNK_STAGES_64:
            if (value != 2 && value != 3) return PMP_EINVAL;
            g_chunk_stages[knob == PMP_KNOB_CHUNK_STAGES_64] = value;
            return PMP_OK;
        case PMP_KNOB_STREAM_SEGMENT:
            if (value != 1 << 17 && value != 1 << 18 && value != 1 << 19) return PMP_EINVAL;
            g_stream_segment = value;
            return PMP_OK;
        default:
            return PMP_EINVAL;
    }
}

int pmp_tune_get(int knob, int *value) {
    if (!value) return PMP_EINVAL;
    switch (knob) {
        case PMP_KNOB_TREE_STAGES_32: *value = g_tree_stages[0]; return PMP_OK;
        case PMP_KNOB_TREE_STAGES_64: *value = g_tree_stages[1]; return PMP_OK;
        case PMP_KNOB_BATCH_P1: *value = g_batch_p1; return PMP_OK;
        case PMP_KNOB_BATCH_SCHED: *value = g_batch_sched; return PMP_OK;
        case PMP_KNOB_BATCH_RANGE: *value = g_batch_range; return PMP_OK;
        case PMP_KNOB_CHUNK_STAGES_32: *value = g_chunk_stages[0]; return PMP_OK;
        case PMP_KNOB_CHUNK_STAGES_64: *value = g_chunk_stages[1]; return PMP_OK;
        case PMP_KNOB_STREAM_SEGMENT: *value = g_stream_segment; return PMP_OK;
        default: return PMP_EINVAL;
    }
}

const char *pmp_strerror(int status) {
    switch (status) {
        case PMP_OK: return "ok";
        case PMP_EINVAL: return "invalid argument";
        case PMP_ENOMEM: return "device allocation failed";
        case PMP_ECUDA: return "CUDA runtime or launch error";
        case PMP_ETOOLONG: return "string needs more than 8 tree levels";
        case PMP_ETIMEOUT: return "bounded device wait ran out";
        case PMP_EALIGN: return "pointer not aligned as required";
        case PMP_ESCRATCH:
            return "input needs more scratch than given (batch: data_bytes too small; "
                   "pmp_hash64_noalloc: the fixed no-allocation buffer)";
        default: return "unknown status";
    }
}

}  // extern "C"
