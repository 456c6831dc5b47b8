// pm_tree.cuh -- one buffer through all levels of the PM+ tree (Algorithm 1)
// in a single persistent launch.
//
// Block roles (6 warps):
//   warps 0-3  consumers: thread r owns level-1 chunk r of the current tile
//              (a tile is 128 level-1 chunks, i.e. one level-2 chunk) and
//              forms its exact sum b_1 + sum a_{1,i} s_i (Sec. 5, eq. 2wlinear)
//              from shared memory with carry-chain multiply-adds on 32-bit
//              limbs, reduces it (Sec. 6.2, Alg. 2) and hands the
//              warp's share of the level-2 sum to the combiner;
//   warp 4     producer: claims tiles from a device work counter and streams
//              each through a ring of S stages of 128 x 128-byte TMA boxes
//              (cp.async.bulk.tensor.2d, 128-byte swizzle, mbarrier);
//   warp 5     combiner: finishes each tile's level-2 value and climbs the
//              tree: the block that completes the last child of a node
//              (atomic arrival counter, no spin-wait) computes the node; the
//              root applies the output step (Sec. 5 end, Sec. 7).
// Consumers never wait for the combiner except through a two-slot ring.
// Streaming updates use two more modes on a buffer of F whole chunks: level-1
// output (consumers write each chunk value, the combiner only waits for the
// end) and level-2 output (tiles are level-2 chunks: the combiner writes the
// value of each complete one and the partial sum of an incomplete last one).
#pragma once
#include <cuda.h>

#include "pm_kernels.cuh"

namespace pm {

struct TreeParams {
    const uint8_t *buf;
    uint64_t len;
    uint64_t F;                   // level-1 chunks made only of string bytes
    uint64_t c[LMAX + 2];         // c[j]: number of chunks of level j (c[levels] == 1)
    int levels;                   // levels applied by Algorithm 1
    Val *vals[LMAX + 2];          // vals[j]: values produced by level j (2 <= j < levels)
    unsigned *ctr[LMAX + 2];      // ctr[j]: arrivals per chunk of level j (3 <= j <= levels)
    unsigned long long *tile_ctr; // work counter (at tile_base when the launch starts); null when one tile
    unsigned long long tile_base; // claims of the counter before this launch (a counter kept across launches)
    const void *key;              // device key, level-major
    void *out;                    // uint32_t / uint64_t
    uint64_t *raw;                // optional (lo, hi) of the tree value
    int use_tma;
    Val *l1_out;                  // level-1 output mode: the F chunk values go here, no combine
    // level-2 output mode (streaming, a segment that starts a level-2 chunk):
    // the values of the complete level-2 chunks (tiles) go to l2_out, the
    // partial sum of an incomplete last tile (or zero) to *l2_part, and when
    // l2_first is set, chunk 0's level-1 value to *l2_first; no climb
    Val *l2_out;
    U192 *l2_part;
    Val *l2_first;
    // let a programmatic dependent launch start once every block's producer
    // has made its last claim (streaming, level-2 mode: the next update's
    // tree launch, which reads nothing this launch writes, overlaps its drain)
    int trigger;
};

constexpr int TREE_CONSUMERS = 128;                  // one level-1 chunk per thread
constexpr int TREE_THREADS = TREE_CONSUMERS + 64;    // + producer warp + combiner warp
constexpr int PRODUCER_TID = TREE_CONSUMERS;
constexpr int COMBINER_WARP = TREE_CONSUMERS / 32 + 1;
constexpr int TILE_ROW_BYTES = 128;                  // TMA box: 128 bytes x 128 rows
constexpr int STAGE_BYTES = TILE_ROW_BYTES * TREE_CONSUMERS;

template <int N, int S>
struct TreeSmem {
    typedef typename Fam<N>::word word;
    static constexpr size_t STAGES = 0;  // 1024-byte aligned for the 128-byte swizzle
    static constexpr size_t KEYS1 = STAGES + (size_t)S * STAGE_BYTES;  // a_{1,1..m}, 16-byte aligned
    static constexpr size_t KEYSALL = KEYS1 + sizeof(word) * M;
    static constexpr size_t BARS = (KEYSALL + sizeof(word) * LMAX * KEY_ROW + 15) / 16 * 16;
    static constexpr size_t PBARS = BARS + 16 * (size_t)S;      // full[S], empty[S]
    static constexpr size_t TILEOF = PBARS + 32;                // pfull[2], pempty[2]
    static constexpr size_t PART = TILEOF + 8 * (size_t)S + 16; // tile of each stage; tile of each part slot
    static constexpr size_t FLAGS = PART + sizeof(U192) * 2 * (TREE_CONSUMERS / 32);
    static constexpr size_t TOTAL = FLAGS + 16;
    static constexpr size_t ALLOC = TOTAL + 1024;  // room to align the base
};

// The last level-1 chunk (index F): string bytes followed by the pad, then
// zeros; computed by one warp from global memory, the value is returned to
// every lane.
template <int N>
__device__ __forceinline__ Val warp_tail_chunk(const TreeParams &P,
                                               const typename Fam<N>::word *keys_l1) {
    const int lane = threadIdx.x & 31;
    const uint64_t W = Fam<N>::W;
    const uint8_t *p = P.buf + P.F * (uint64_t)M * W;
    const uint64_t rem = P.len - P.F * (uint64_t)M * W;  // < m W string bytes
    U192 acc = {0, 0, 0};
#pragma unroll
    for (int q = 0; q < M / 32; ++q) {
        const int i = lane + 32 * q;  // word index in the chunk
        Val s = {0, 0};
        if constexpr (N == 32) {
            const uint64_t unit = load_unit_padded(p, rem, (uint64_t)(i >> 1));
            s.lo = (i & 1) ? (unit >> 32) : (unit & 0xffffffffull);
        } else {
            s.lo = load_unit_padded(p, rem, (uint64_t)i);
        }
        mac(acc, keys_l1[1 + i], s);
    }
    acc = warp_sum192(acc);
    Val v = {0, 0};
    if (lane == 0) {
        add192(acc, (uint64_t)keys_l1[0], 0, 0);
        v = reduce<N>(acc);
    }
    v.lo = __shfl_sync(0xffffffffu, v.lo, 0);
    v.hi = __shfl_sync(0xffffffffu, v.hi, 0);
    return v;
}

// PM+64 tiles are read as rows of half a chunk (512 bytes apart, as PM+32's
// whole chunks are): a 1 KiB-stride column of 128 chunks reached HBM
// measurably slower than two 512-byte-stride halves.
template <int N> __host__ __device__ constexpr bool half_rows() { return N == 64; }
template <int N> constexpr bool HALF_ROWS = half_rows<N>();

// The exact sum of this lane's accumulator and that of lane ^ 1.
__device__ __forceinline__ void add_pair_lane(AccC64 &a) {
    AccC64 o;
    o.r0 = __shfl_xor_sync(0xffffffffu, a.r0, 1);
    o.r1 = __shfl_xor_sync(0xffffffffu, a.r1, 1);
    o.r2 = __shfl_xor_sync(0xffffffffu, a.r2, 1);
    o.r3 = __shfl_xor_sync(0xffffffffu, a.r3, 1);
    o.r4 = __shfl_xor_sync(0xffffffffu, a.r4, 1);
    o.x0 = __shfl_xor_sync(0xffffffffu, a.x0, 1);
    o.x1 = __shfl_xor_sync(0xffffffffu, a.x1, 1);
    o.x2 = __shfl_xor_sync(0xffffffffu, a.x2, 1);
    a.merge(o);
}

// Consumers of the half-row layout (n = 64). A tile of 128 chunks is 256
// half-rows; stage c holds column c % 4 (128 bytes) of half-rows
// 128 (c / 4) .. + 127, so thread r reads half r & 1 of chunk
// 64 (c / 4) + r / 2. Lanes r and r ^ 1 add their exact sums after each group
// of four stages; the even lane keeps the chunk's value. Otherwise as the
// whole-row consumers of k_tree: level-1 values (streaming level-1 mode), the
// first value, the tail chunk, the single chunk of a one-level string, and
// each warp's share of the level-2 sum for the combiner.
template <int N, int S>
__device__ __forceinline__ void consume_half_rows(const TreeParams &P, const uint8_t *stages, const uint4 *keys1,
                                                  const typename Fam<N>::word *keysall, uint64_t *full,
                                                  uint64_t *empty, uint64_t *pfull, uint64_t *pempty,
                                                  volatile int64_t *tile_of, volatile int64_t *part_tile,
                                                  U192 *part, volatile int *abort_flag) {
    typedef typename AccCT<N>::t Acc;
    constexpr int NC = M * Fam<N>::W / TILE_ROW_BYTES;  // 8 stages per tile
    constexpr int HALF_GROUPS = M * Fam<N>::W / 2 / 16;  // 16-byte key groups per half chunk
    const int r = threadIdx.x, warp = r >> 5, lane = r & 31, h = r & 1;
    const bool own = h == 0;  // the even lane of a pair keeps the chunk's value
    // the tail chunk (index F): tile F / 128, group (F % 128) / 64, even lane 2 (F % 64)
    const uint64_t tail_tile = P.F / TREE_CONSUMERS;
    const int tail_g = (int)((P.F % TREE_CONSUMERS) / 64);
    const int tail_r = (int)(2 * (P.F % 64));
    uint32_t it = 0, tseq = 0;
    for (;;) {
        uint32_t s = it % S, ph = (it / S) & 1;
        mbar_wait(&full[s], ph, abort_flag);
        const int64_t t = tile_of[s];
        if (t < 0 || *abort_flag) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            ++it;
            break;
        }
        const uint64_t cbase = (uint64_t)t * TREE_CONSUMERS + (uint64_t)(r >> 1);  // chunk of group 0
        const bool has_data = P.use_tma && (uint64_t)t * TREE_CONSUMERS < P.F;
        Val v0 = {0, 0}, v1 = {0, 0};  // values of the chunks of groups 0 and 1 (even lanes)
        Acc acc0, acc1;  // two independent accumulator sets (even / odd 16-byte groups)
        for (int c = 0; c < NC; ++c, ++it) {
            const int g = c / 4, cc = c % 4;
            if (cc == 0) {
                acc0.zero();
                acc1.zero();
            }
            if (c > 0) {
                s = it % S;
                ph = (it / S) & 1;
                mbar_wait(&full[s], ph, abort_flag);
            }
            const uint64_t chunk = cbase + 64 * (uint64_t)g;
            if (has_data && chunk < P.F) {
                const uint8_t *row = stages + (size_t)s * STAGE_BYTES + r * TILE_ROW_BYTES;
                const uint4 *k = keys1 + h * HALF_GROUPS + cc * 8;
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    // 128-byte swizzle: unit j of row r sits at unit j ^ (r mod 8)
                    const uint4 d0 = *reinterpret_cast<const uint4 *>(row + ((j ^ (r & 7)) << 4));
                    const uint4 d1 = *reinterpret_cast<const uint4 *>(row + (((j + 1) ^ (r & 7)) << 4));
                    add16c(acc0, k[j], d0);
                    add16c(acc1, k[j + 1], d1);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            if (cc == 3) {  // the group's chunks: both halves
                acc0.merge(acc1);
                add_pair_lane(acc0);
                if (own && chunk < P.F) {
                    const Val x = acc0.finish((uint64_t)keysall[0]);
                    if (g == 0)
                        v0 = x;
                    else
                        v1 = x;
                }
            }
        }
        const uint64_t ch0 = cbase, ch1 = cbase + 64;
        if (P.l1_out) {  // streaming: whole chunks only, their values for the level folds
            if (own) {
                if (ch0 < P.F) P.l1_out[ch0] = v0;
                if (ch1 < P.F) P.l1_out[ch1] = v1;
            }
            continue;
        }
        if (P.l2_first && own && ch0 == 0) *P.l2_first = v0;
        if ((uint64_t)t == tail_tile && warp == tail_r / 32 && !P.l2_out) {
            const Val vt = warp_tail_chunk<N>(P, keysall);
            if (r == tail_r) {
                if (tail_g == 0)
                    v0 = vt;
                else
                    v1 = vt;
            }
        }
        if (P.levels == 1) {  // one chunk in all: it is the hash
            if (own && ch0 == 0) write_output<N>(P.out, P.raw, 0, v0);
            continue;
        }
        // this warp's share of the level-2 sum of chunk t: sum a_{2,i+1} v_i
        U192 prod = {0, 0, 0};
        if (own) {
            if (ch0 < P.c[1]) mac(prod, keysall[KEY_ROW + 1 + (r >> 1)], v0);
            if (ch1 < P.c[1]) mac(prod, keysall[KEY_ROW + 1 + 64 + (r >> 1)], v1);
        }
        prod = warp_sum192(prod);
        const uint32_t ps = tseq & 1, pph = (tseq >> 1) & 1;
        ++tseq;
        if (lane == 0) {
            mbar_wait(&pempty[ps], pph ^ 1, abort_flag);
            part[ps * 4 + warp] = prod;
            if (warp == 0) part_tile[ps] = t;
            mbar_arrive(&pfull[ps]);
        }
    }
    // tell the combiner there are no more tiles
    const uint32_t ps = tseq & 1, pph = (tseq >> 1) & 1;
    if (lane == 0) {
        mbar_wait(&pempty[ps], pph ^ 1, abort_flag);
        if (warp == 0) part_tile[ps] = -1;
        mbar_arrive(&pfull[ps]);
    }
}

template <int N, int S>
__global__ void __launch_bounds__(TREE_THREADS)
    k_tree(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ TreeParams P) {
    typedef typename Fam<N>::word word;
    typedef TreeSmem<N, S> L;
    typedef typename AccCT<N>::t Acc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>(
        (reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~(uintptr_t)1023);
    uint8_t *stages = smem + L::STAGES;
    word *keys1w = reinterpret_cast<word *>(smem + L::KEYS1);
    const uint4 *keys1 = reinterpret_cast<const uint4 *>(keys1w);  // key words of 16-byte unit u
    word *keysall = reinterpret_cast<word *>(smem + L::KEYSALL);
    uint64_t *full = reinterpret_cast<uint64_t *>(smem + L::BARS);
    uint64_t *empty = full + S;
    uint64_t *pfull = reinterpret_cast<uint64_t *>(smem + L::PBARS);
    uint64_t *pempty = pfull + 2;
    volatile int64_t *tile_of = reinterpret_cast<volatile int64_t *>(smem + L::TILEOF);
    volatile int64_t *part_tile = tile_of + S;
    U192 *part = reinterpret_cast<U192 *>(smem + L::PART);  // [2][4]
    volatile int *abort_flag = reinterpret_cast<volatile int *>(smem + L::FLAGS);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const word *gkey = static_cast<const word *>(P.key);
    for (int i = tid; i < LMAX * KEY_ROW; i += TREE_THREADS) keysall[i] = gkey[i];
    for (int i = tid; i < M; i += TREE_THREADS) keys1w[i] = gkey[1 + i];
    if (tid == PRODUCER_TID) {
        for (int s = 0; s < S; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], TREE_CONSUMERS / 32);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&pfull[s], TREE_CONSUMERS / 32);
            mbar_init(&pempty[s], 1);
        }
        *abort_flag = 0;
        fence_barrier_init();
    }
    __syncthreads();

    const uint64_t ntiles = P.levels >= 2 ? P.c[2] : 1;
    constexpr int NC = M * Fam<N>::W / TILE_ROW_BYTES;  // column stages per tile

    if (warp == PRODUCER_TID / 32) {
        // ---------------- producer: claims tiles, issues TMA loads -----------
        if (lane != 0) return;
        if (P.use_tma) prefetch_tmap(&tmap);
        uint32_t it = 0, issued_mask = 0, last_par = 0;
        uint64_t next_static = 0;
        for (;;) {
            uint64_t t;
            if (P.tile_ctr)
                t = atomicAdd(P.tile_ctr, 1ull) - P.tile_base;
            else
                t = next_static++;
            const bool done = t >= ntiles || *abort_flag;
            const bool data = !done && P.use_tma && t * TREE_CONSUMERS < P.F;
            const int nslots = done ? 1 : NC;
            for (int c = 0; c < nslots; ++c, ++it) {
                const uint32_t s = it % S, ph = (it / S) & 1;
                mbar_wait(&empty[s], ph ^ 1, abort_flag);
                tile_of[s] = done ? -1 : (int64_t)t;
                if (data) {
                    mbar_arrive_expect_tx(&full[s], STAGE_BYTES);
                    if constexpr (HALF_ROWS<N>)  // column c % 4 of half-rows 128 (c / 4) .. + 127
                        tma_load_2d(stages + (size_t)s * STAGE_BYTES, &tmap, (c % 4) * TILE_ROW_BYTES,
                                    (int)(t * 2 * TREE_CONSUMERS + (c / 4) * TREE_CONSUMERS), &full[s]);
                    else
                        tma_load_2d(stages + (size_t)s * STAGE_BYTES, &tmap, c * TILE_ROW_BYTES,
                                    (int)(t * TREE_CONSUMERS), &full[s]);
                    issued_mask |= 1u << s;
                    last_par = (last_par & ~(1u << s)) | (ph << s);
                } else {
                    mbar_arrive(&full[s]);
                }
            }
            if (done) break;
        }
        if (P.trigger) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
        if (*abort_flag) {
            // let the copies already issued land before the block can exit
            volatile int no_abort = 0;
            for (int s = 0; s < S; ++s)
                if (issued_mask & (1u << s)) mbar_wait(&full[s], (last_par >> s) & 1, &no_abort);
        }
        return;
    }

    if (warp == COMBINER_WARP) {
        // ---------------- combiner: level 2 of each tile, then the climb ------
        for (uint32_t tseq = 0;; ++tseq) {
            const uint32_t ps = tseq & 1, pph = (tseq >> 1) & 1;
            mbar_wait(&pfull[ps], pph, abort_flag);
            const int64_t t = part_tile[ps];
            U192 sum = part[ps * 4];
            add192(sum, part[ps * 4 + 1]);
            add192(sum, part[ps * 4 + 2]);
            add192(sum, part[ps * 4 + 3]);
            __syncwarp();
            if (lane == 0) mbar_arrive(&pempty[ps]);
            if (t < 0 || *abort_flag) break;
            if (P.l2_out) {
                if (lane == 0) {
                    const bool whole = (uint64_t)(t + 1) * M <= P.c[1];
                    if (whole) {
                        U192 x = sum;
                        add192(x, (uint64_t)keysall[KEY_ROW], 0, 0);  // b_2
                        P.l2_out[t] = reduce<N>(x);
                    }
                    if ((uint64_t)t + 1 == P.c[2]) *P.l2_part = whole ? U192{0, 0, 0} : sum;
                }
                continue;
            }
            Val w = {0, 0};
            if (lane == 0) {
                add192(sum, (uint64_t)keysall[KEY_ROW], 0, 0);  // b_2
                w = reduce<N>(sum);
            }
            int j = 2;
            uint64_t node = (uint64_t)t;
            for (;;) {
                if (j == P.levels) {
                    if (lane == 0) write_output<N>(P.out, P.raw, 0, w);
                    break;
                }
                const uint64_t q = node / M;
                unsigned last = 0;
                if (lane == 0) {
                    P.vals[j][node] = w;
                    __threadfence();
                    const uint64_t left = P.c[j] - q * M;
                    const unsigned expect = (unsigned)(left < (uint64_t)M ? left : (uint64_t)M);
                    last = (atomicAdd(&P.ctr[j + 1][q], 1u) + 1 == expect);
                }
                if (!__shfl_sync(0xffffffffu, last, 0)) break;
                __threadfence();
                U192 pr = {0, 0, 0};
#pragma unroll
                for (int k = 0; k < M / 32; ++k) {
                    const uint64_t idx = q * M + lane + 32 * k;
                    if (idx < P.c[j]) {
                        Val x;
                        x.lo = __ldcg(reinterpret_cast<const unsigned long long *>(&P.vals[j][idx].lo));
                        x.hi = __ldcg(reinterpret_cast<const unsigned long long *>(&P.vals[j][idx].hi));
                        mac(pr, keysall[j * KEY_ROW + 1 + lane + 32 * k], x);
                    }
                }
                pr = warp_sum192(pr);
                if (lane == 0) {
                    add192(pr, (uint64_t)keysall[j * KEY_ROW], 0, 0);
                    w = reduce<N>(pr);
                }
                ++j;
                node = q;
            }
        }
        // a programmatic dependent (a level-2 mode launch after another one)
        // ends only after the launch before it: work that follows it on the
        // stream then also follows that launch
        if (P.trigger) asm volatile("griddepcontrol.wait;" ::: "memory");
        return;
    }

    // ---------------- consumers: thread r owns row r of each tile -------------
    const int r = tid;
    if constexpr (HALF_ROWS<N>) {
        consume_half_rows<N, S>(P, stages, keys1, keysall, full, empty, pfull, pempty, tile_of, part_tile, part,
                                abort_flag);
        return;
    }
    const uint64_t tail_tile = P.F / TREE_CONSUMERS;
    const int tail_warp = (int)((P.F % TREE_CONSUMERS) / 32);
    uint32_t it = 0, tseq = 0;
    for (;;) {
        uint32_t s = it % S, ph = (it / S) & 1;
        mbar_wait(&full[s], ph, abort_flag);
        const int64_t t = tile_of[s];
        if (t < 0 || *abort_flag) {
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
            ++it;
            break;
        }
        const uint64_t chunk = (uint64_t)t * TREE_CONSUMERS + r;
        const bool has_data = P.use_tma && (uint64_t)t * TREE_CONSUMERS < P.F;
        Acc acc0, acc1;  // two independent accumulator sets (even / odd units)
        acc0.zero();
        acc1.zero();
        for (int c = 0; c < NC; ++c, ++it) {
            if (c > 0) {
                s = it % S;
                ph = (it / S) & 1;
                mbar_wait(&full[s], ph, abort_flag);
            }
            if (has_data && chunk < P.F) {
                const uint8_t *row = stages + (size_t)s * STAGE_BYTES + r * TILE_ROW_BYTES;
#pragma unroll
                for (int j = 0; j < 8; j += 2) {
                    // 128-byte swizzle: unit j of row r sits at unit j ^ (r mod 8)
                    const uint4 d0 = *reinterpret_cast<const uint4 *>(row + ((j ^ (r & 7)) << 4));
                    const uint4 d1 = *reinterpret_cast<const uint4 *>(row + (((j + 1) ^ (r & 7)) << 4));
                    add16c(acc0, keys1[c * 8 + j], d0);
                    add16c(acc1, keys1[c * 8 + j + 1], d1);
                }
            }
            __syncwarp();
            if (lane == 0) mbar_arrive(&empty[s]);
        }
        Val v = {0, 0};
        if (chunk < P.F) {
            acc0.merge(acc1);
            v = acc0.finish((uint64_t)keysall[0]);
        }
        if (P.l1_out) {  // streaming: whole chunks only, their values for the level folds
            if (chunk < P.F) P.l1_out[chunk] = v;
            continue;
        }
        if (P.l2_first && chunk == 0) *P.l2_first = v;
        if ((uint64_t)t == tail_tile && warp == tail_warp && !P.l2_out) {
            const Val vt = warp_tail_chunk<N>(P, keysall);
            if (chunk == P.F) v = vt;
        }
        if (P.levels == 1) {  // one chunk in all: it is the hash
            if (chunk == 0) write_output<N>(P.out, P.raw, 0, v);
            continue;
        }
        // this warp's share of the level-2 sum of chunk t: sum a_{2,r+1} v_r
        U192 prod = {0, 0, 0};
        if (chunk < P.c[1]) mac(prod, keysall[KEY_ROW + 1 + r], v);
        prod = warp_sum192(prod);
        const uint32_t ps = tseq & 1, pph = (tseq >> 1) & 1;
        ++tseq;
        if (lane == 0) {
            mbar_wait(&pempty[ps], pph ^ 1, abort_flag);
            part[ps * 4 + warp] = prod;
            if (warp == 0) part_tile[ps] = t;
            mbar_arrive(&pfull[ps]);
        }
    }
    // tell the combiner there are no more tiles
    const uint32_t ps = tseq & 1, pph = (tseq >> 1) & 1;
    if (lane == 0) {
        mbar_wait(&pempty[ps], pph ^ 1, abort_flag);
        if (warp == 0) part_tile[ps] = -1;
        mbar_arrive(&pfull[ps]);
    }
}

}  // namespace pm
