// pm_range.cuh -- ragged batch of strings, sorted by length inside ranges.
//
// Each block of k_batch_range takes ranges of C::RS consecutive strings,
// claimed from a device counter one range ahead (the offsets of the next
// range, and then its first bytes, are prefetched into L2 while the current
// one is hashed). Thread t owns strings t, t + C::THREADS, ... of a range,
// whose offsets it reads coalesced into registers. A range is hashed in
// fills: a fill is the longest run of strings [x, y) whose bytes span at most
// C::CAP bytes (16-byte aligned), staged in shared memory by one bulk copy
// (cp.async.bulk, completing on an mbarrier); a string too long for any fill
// forms a fill of its own and is read from global memory. For each fill the
// block
//   1. sorts the fill's one-chunk strings (fewer than m words once padded,
//      Sec. 4) by their count of whole 8-byte units, while the copy is in
//      flight: a counting sort in shared memory, longest class first, so that
//      the 32 strings of a warp group have nearly the same length and the
//      unit loop keeps every lane busy;
//   2. lets warps claim work: the fill's strings of 2..BIG_CHUNKS-1 chunks
//      and, for n = 64, its one-chunk strings of RG_WIDE_UNITS or more
//      whole units first (one warp per string, from global memory: one or
//      two levels of Algorithm 1), then the groups of 32 sorted strings. In a group, lane l
//      forms b_1 + sum_i a_{1,i} s_i of its string (Sec. 5, eq. 2wlinear)
//      from shared memory with carry-chain multiply-adds (the key words of a
//      unit position are the same for every lane: a shared-memory
//      broadcast), adds the tail unit (last bytes + the 0x01 pad of Sec. 4),
//      reduces (Sec. 6.2, Algorithm 2) and applies the output step (Sec. 5,
//      Sec. 7).
// Strings of BIG_CHUNKS chunks or more are queued for the chunk kernel
// (pm_long.cuh), which runs as a programmatic dependent of this kernel.
#pragma once
#include "pm_lane.cuh"

namespace pm {

// A launch configuration of the kernel: THREADS per block, R strings per
// range (R / THREADS per thread), CAP staged bytes per fill, BLOCKS resident
// blocks per SM (what the shared memory and registers of a block allow).
template <int T, int R, int CAPK, int BPS>
struct RangeCfg {
    static constexpr int THREADS = T, WARPS = T / 32, RS = R, SPT = R / T, BLOCKS = BPS;
    static constexpr uint32_t CAP = (uint32_t)CAPK * 1024, PREFETCH = CAP;
    static_assert(R % T == 0 && CAP < 65536, "staging addresses are kept in 16 bits");
};
typedef RangeCfg<256, 1024, 56, 3> RangeWide;   // 8 warps a block, 3 blocks per SM
typedef RangeCfg<128, 512, 28, 6> RangeNarrow;  // 4 warps a block, 6 blocks per SM

// One-chunk strings of at least this many whole units are hashed by a whole
// warp (n = 64 only: an n = 32 chunk has 64 units), so that no lane of a
// sorted group runs a serial chain of more than 63 units.
constexpr int RG_WIDE_UNITS = 64;

// Units of one level-1 chunk (m words): the sort classes of one-chunk strings.
template <int N>
__host__ __device__ constexpr int range_classes() {
    return M * Fam<N>::W / 8;
}

template <int N, class C>
struct RangeSmem {
    uint8_t data[C::CAP];                           // the fill's bytes (16-byte aligned)
    uint2 rec[C::RS];                                // [0, total): sorted (string, addr | len << 16);
                                                    // from the top: multi-chunk strings of the fill
    uint32_t cls[range_classes<N>()];               // class counts, then first positions
    alignas(16) typename UnitKey<N>::t ku[range_classes<N>()];  // a_{1,i} of the words of unit u
    typename Fam<N>::word keys2[KEY_ROW];           // b_2, a_{2,1..m}
    int64_t src;                                    // first staged byte of the fill (16-byte aligned)
    int64_t rend;                                   // end of the range's last string
    uint64_t bar;                                   // mbarrier of a fill's copy
    uint32_t y, nmed, total, work, next;
    int abort;
};

template <int N, class C>
constexpr size_t range_smem_bytes() {
    return sizeof(RangeSmem<N, C>);
}

__device__ __forceinline__ uint64_t lds64(const uint8_t *p) { return *reinterpret_cast<const uint64_t *>(p); }

// The exact value of a carry-chain accumulator as a three-word integer.
__device__ __forceinline__ U192 exact(const AccC32 &a) {
    U192 s = {(uint64_t)a.r0 | ((uint64_t)a.r1 << 32), (uint64_t)a.r2, 0};
    return s;
}
__device__ __forceinline__ U192 exact(const AccC64 &a) {
    U192 s = {(uint64_t)a.r0 | ((uint64_t)a.r1 << 32), (uint64_t)a.r2 | ((uint64_t)a.r3 << 32), (uint64_t)a.r4};
    add192(s, (uint64_t)a.x0 << 32, (uint64_t)a.x1 | ((uint64_t)a.x2 << 32), 0);
    return s;
}

// Wait for a fill's copy, sleeping in hardware between checks; bounded by
// WAIT_LIMIT_NS (then PMP_ETIMEOUT is recorded, the block's other threads
// give up at once, and a copy still in flight gets one more bounded wait).
__device__ __forceinline__ bool wait_copies(uint64_t *bar, uint32_t parity, int *abort, int *call_status) {
    const uint64_t t0 = globaltimer_ns();
    while (!mbar_try_wait_hint(bar, parity, 1000000u)) {
        if (*(volatile int *)abort) return false;
        if (globaltimer_ns() - t0 > WAIT_LIMIT_NS) {
            record_status(call_status, STATUS_TIMEOUT);
            *(volatile int *)abort = 1;
            const uint64_t t1 = globaltimer_ns();
            while (!mbar_try_wait(bar, parity) && globaltimer_ns() - t1 < WAIT_LIMIT_NS) {
            }
            return false;
        }
    }
    return true;
}

__device__ __forceinline__ int64_t align16_down(int64_t x) { return x & ~(int64_t)15; }
__device__ __forceinline__ int64_t align16_up(int64_t x) { return (x + 15) & ~(int64_t)15; }

// One string hashed by a whole warp: a one-chunk string of at least
// RG_WIDE_UNITS whole units, or one of 2..BIG_CHUNKS-1 chunks. Chunk c's
// value v_c = (b_1 + sum_i a_{1,i} s_{mc+i}) mod p, lane l on units l, l + 32,
// ... of the chunk (the next chunk's loads in flight); with one chunk v_0 is
// the hash, else h = (b_2 + sum_c a_{2,c+1} v_c) mod p, the level-2 chunk
// being the root (Algorithm 1). The bytes are read from global memory (a
// test that read them from the staged fill instead measured slower).
template <int N, class Sm>
__device__ __forceinline__ void range_medium(const BatchParams &P, const Sm &S, int64_t i, const uint8_t *p,
                                             uint64_t len, uint64_t b1) {
    typedef typename AccCT<N>::t AccC;
    constexpr int UPL = range_classes<N>() / 32;  // units per lane per chunk: 2 or 4
    constexpr uint64_t CB = (uint64_t)M * Fam<N>::W;
    const int lane = threadIdx.x & 31;
    const uint64_t c1 = (len / Fam<N>::W + M) / M;  // ceil((len / W + 1) / m)
    const uint64_t full = len / CB;                 // chunks of string bytes only
    auto load = [&](uint64_t c, uint64_t (&x)[UPL]) {
        const uint8_t *cp = p + c * CB;
#pragma unroll
        for (int q = 0; q < UPL; ++q) {
            const uint64_t u = (uint64_t)(lane + 32 * q);
            x[q] = c < full ? __ldg(reinterpret_cast<const unsigned long long *>(cp) + u)
                            : load_unit_padded(cp, len - c * CB, u);
        }
    };
    uint64_t x[UPL], y[UPL];
    load(0, x);
    U192 s2 = {0, 0, 0};
    Val v = {0, 0};
    for (uint64_t c = 0; c < c1; ++c) {
        if (c + 1 < c1) load(c + 1, y);
        AccC a;
        a.zero();
#pragma unroll
        for (int q = 0; q < UPL; ++q) add_unit_c(a, S.ku[lane + 32 * q], x[q]);
        U192 t = warp_sum192(exact(a));
        if (lane == 0) {
            add192(t, b1, 0, 0);
            v = reduce<N>(t);
            mac(s2, S.keys2[1 + c], v);
        }
#pragma unroll
        for (int q = 0; q < UPL; ++q) x[q] = y[q];
    }
    if (lane == 0) {
        add192(s2, (uint64_t)S.keys2[0], 0, 0);
        store_result<N>(P, i, c1 == 1 ? v : reduce<N>(s2));
    }
}

// Sorted record k of a fill: string j of the range, its first byte in the
// staged fill and its length.
template <int N, class C>
__device__ __forceinline__ void rec_entry(const RangeSmem<N, C> &S, uint32_t k, uint32_t &j, uint32_t &addr,
                                          uint32_t &len) {
    const uint2 r = S.rec[k];
    j = r.x;
    addr = r.y & 0xffffu;
    len = r.y >> 16;
}

// Group of up to 32 sorted one-chunk strings rec[k0 ..], whole warp, lane l
// on string k0 + l. Sorted longest first: lane 0 has the most whole units,
// the last active lane the fewest.
template <int N, class Sm>
__device__ __forceinline__ void range_group(const BatchParams &P, const Sm &S, int64_t s0, uint32_t k0,
                                            uint32_t total, uint64_t b1) {
    typedef typename AccCT<N>::t AccC;
    typedef typename UnitKey<N>::t KW;
    const int lane = threadIdx.x & 31;
    const uint32_t nact = total - k0 < 32u ? total - k0 : 32u;
    const bool act = (uint32_t)lane < nact;
    uint32_t rj, raddr, rlen;
    rec_entry(S, k0 + (act ? lane : 0), rj, raddr, rlen);
    const uint32_t len = act ? rlen : 0u;
    const uint32_t full = len >> 3;
    const uint32_t fmax = __shfl_sync(0xffffffffu, full, 0);
    const uint32_t fmin = __shfl_sync(0xffffffffu, full, nact - 1);
    const uint8_t *p = S.data + raddr;
    const uint4 *kp = reinterpret_cast<const uint4 *>(S.ku);  // key words of units 2v, 2v + 1
    AccC acc;
    acc.zero();
    uint32_t u = 0;
#pragma unroll 1
    for (; u + 4 <= fmin; u += 4) {
        const uint64_t x0 = lds64(p + 8 * u), x1 = lds64(p + 8 * u + 8), x2 = lds64(p + 8 * u + 16),
                       x3 = lds64(p + 8 * u + 24);
        const uint4 ka = kp[u / 2], kb = kp[u / 2 + 1];
        KW k0w, k1w, k2w, k3w;
        if constexpr (N == 32) {
            k0w = make_uint2(ka.x, ka.y);
            k1w = make_uint2(ka.z, ka.w);
            k2w = make_uint2(kb.x, kb.y);
            k3w = make_uint2(kb.z, kb.w);
        } else {
            k0w = (uint64_t)ka.x | ((uint64_t)ka.y << 32);
            k1w = (uint64_t)ka.z | ((uint64_t)ka.w << 32);
            k2w = (uint64_t)kb.x | ((uint64_t)kb.y << 32);
            k3w = (uint64_t)kb.z | ((uint64_t)kb.w << 32);
        }
        add_unit_c(acc, k0w, x0);
        add_unit_c(acc, k1w, x1);
        add_unit_c(acc, k2w, x2);
        add_unit_c(acc, k3w, x3);
    }
#pragma unroll 1
    for (; u < fmax; ++u)
        if (u < full) add_unit_c(acc, S.ku[u], lds64(p + 8 * u));
    const uint64_t tw = (len & 7) ? lds64(p + 8 * full) : 0ull;
    add_unit_c(acc, S.ku[full], tail_unit(tw, len));
    if (act) store_result<N>(P, s0 + (int64_t)rj, acc.finish(b1));
}

template <int N, class C>
__global__ void __launch_bounds__(C::THREADS, C::BLOCKS) k_batch_range(const __grid_constant__ BatchParams P) {
    typedef typename Fam<N>::word word;
    typedef RangeSmem<N, C> Sm;
    constexpr int NCLS = range_classes<N>();
    constexpr int64_t CB = (int64_t)M * Fam<N>::W;  // bytes of a level-1 chunk
    extern __shared__ __align__(128) uint8_t smem_raw[];
    Sm &S = *reinterpret_cast<Sm *>(smem_raw);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // the chunk kernel, when it follows (big_cap > 0), may be scheduled now: it
    // waits for this grid's results; otherwise nothing may start early
    if (P.big_cap) asm volatile("griddepcontrol.launch_dependents;" ::: "memory");
    const word *gkey = static_cast<const word *>(P.key);
    for (int u = tid; u < NCLS; u += C::THREADS) S.ku[u] = unit_key<N>(gkey, u);
    for (int i = tid; i < KEY_ROW; i += C::THREADS) S.keys2[i] = gkey[KEY_ROW + i];
    if (tid == 0) {
        S.abort = 0;
        mbar_init(&S.bar, 1);
        fence_barrier_init();
    }
    const uint64_t b1 = (uint64_t)gkey[0];
    const uint32_t nranges = (uint32_t)((P.n + C::RS - 1) / C::RS);
    uint32_t phase = 0;
    uint32_t range = blockIdx.x;
    while (range < nranges) {
        const int64_t s0 = (int64_t)range * C::RS;
        const int cnt = (int)(P.n - s0 < C::RS ? P.n - s0 : C::RS);
        if (tid == 0) S.next = gridDim.x + atomicAdd(P.tile_ctr, 1u);
        // strings j = tid + C::THREADS q: span [st, en), class (whole units)
        int64_t st[C::SPT], en[C::SPT];
        uint32_t cls[C::SPT];  // whole 8-byte units of a one-chunk string; NCLS otherwise
#pragma unroll
        for (int q = 0; q < C::SPT; ++q) {
            const int j = tid + C::THREADS * q;
            const bool valid = j < cnt;
            const int64_t o = valid ? __ldg(P.off + s0 + j) : 0;
            en[q] = valid ? __ldg(P.off + s0 + j + 1) : 0;
            st[q] = (o + 7) & ~(int64_t)7;
            const int64_t l = en[q] - st[q];
            cls[q] = valid && l >= 0 && (l >> 3) < RG_WIDE_UNITS && l < CB ? (uint32_t)(l >> 3) : (uint32_t)NCLS;
        }
        // the first fill's start and the range's end: when the whole range
        // fits the buffer, its one fill needs no fit test
        if (tid == 0) {
            S.src = align16_down(st[0]);
            S.y = (uint32_t)cnt;
            S.nmed = 0;
            S.work = 0;
        }
#pragma unroll
        for (int q = 0; q < C::SPT; ++q)
            if (tid + C::THREADS * q == cnt - 1) S.rend = en[q];
        for (int c = tid; c < NCLS; c += C::THREADS) S.cls[c] = 0;
        __syncthreads();  // S.next is set; the previous range is done with shared memory
        const uint32_t next = S.next;
        if (next < nranges) {  // the next range's offsets into L2, a line per thread
            const int64_t ns0 = (int64_t)next * C::RS;
            const int64_t nend = P.n - ns0 < C::RS ? P.n : ns0 + C::RS;
            const int64_t k = ns0 + 16 * tid;
            if (k <= nend) prefetch_l2(P.off + k);
        }
        int x = 0;  // first string of the fill
        bool first_fill = true;
        while (x < cnt) {
            if (!first_fill) {
#pragma unroll
                for (int q = 0; q < C::SPT; ++q)
                    if (tid + C::THREADS * q == x) S.src = align16_down(st[q]);
                if (tid == 0) {
                    S.y = (uint32_t)cnt;
                    S.nmed = 0;
                    S.work = 0;
                }
                for (int c = tid; c < NCLS; c += C::THREADS) S.cls[c] = 0;
                __syncthreads();
            }
            const int64_t src = S.src;
            if (!first_fill || align16_up(S.rend) - src > (int64_t)C::CAP) {
                // the fill ends before the first string whose bytes reach past the buffer
#pragma unroll
                for (int q = 0; q < C::SPT; ++q) {
                    const int j = tid + C::THREADS * q;
                    if (j >= x && j < cnt && align16_up(en[q]) - src > (int64_t)C::CAP) {
                        atomicMin(&S.y, (uint32_t)j);
                        break;
                    }
                }
                __syncthreads();
            }
            int y = (int)S.y;
            const bool staged = y > x;  // else string x alone is too long: read from global
            if (!staged) y = x + 1;
            uint32_t rank[C::SPT];
#pragma unroll
            for (int q = 0; q < C::SPT; ++q) {
                const int j = tid + C::THREADS * q;
                const bool in = j >= x && j < y;
                rank[q] = 0;
                if (in && staged && j == y - 1) {  // the fill's last string copies the fill
                    const uint32_t bytes = (uint32_t)(align16_up(en[q]) - src);
                    mbar_arrive_expect_tx(&S.bar, bytes);
                    bulk_load(S.data, P.base + src, bytes, &S.bar);
                }
                // rank among the strings of its class (a warp-aggregated form
                // with __match_any_sync measured slower)
                const bool one = in && cls[q] < (uint32_t)NCLS;
                if (one) rank[q] = atomicAdd(&S.cls[cls[q]], 1u);
                bool big = false;
                if (in && !one) {  // a wide one-chunk string or a longer one
                    const uint64_t l = (uint64_t)(en[q] - st[q]);
                    big = l / Fam<N>::W + 1 > (uint64_t)M * (BIG_CHUNKS - 1);
                    if (!big) S.rec[C::RS - 1 - atomicAdd(&S.nmed, 1u)].x = (uint32_t)j;
                }
                const unsigned bb = __ballot_sync(0xffffffffu, big);
                if (bb) reserve_big<N>(P, bb, s0 + j, big ? (uint64_t)(en[q] - st[q]) : 0);
            }
            if (!staged && tid == 0) mbar_arrive(&S.bar);  // no copy: the phase completes now
            __syncthreads();
            if (warp == 0) {
                // first position of each class, longest class first
                constexpr int PER = NCLS / 32;
                uint32_t v[PER], s = 0;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    v[i] = S.cls[NCLS - 1 - (lane * PER + i)];
                    s += v[i];
                }
                uint32_t incl = s;
#pragma unroll
                for (int d = 1; d < 32; d <<= 1) {
                    const uint32_t t = __shfl_up_sync(0xffffffffu, incl, d);
                    if (lane >= d) incl += t;
                }
                uint32_t pos = incl - s;
#pragma unroll
                for (int i = 0; i < PER; ++i) {
                    S.cls[NCLS - 1 - (lane * PER + i)] = pos;
                    pos += v[i];
                }
                if (lane == 31) S.total = incl;
            }
            __syncthreads();
#pragma unroll
            for (int q = 0; q < C::SPT; ++q) {
                const int j = tid + C::THREADS * q;
                if (j >= x && j < y && cls[q] < (uint32_t)NCLS) {
                    const uint32_t addr = (uint32_t)(st[q] - src), len = (uint32_t)(en[q] - st[q]);
                    S.rec[S.cls[cls[q]] + rank[q]] = make_uint2((uint32_t)j, addr | (len << 16));
                }
            }
            __syncthreads();
            if (first_fill && tid == 0 && next < nranges) {
                // the next range's first bytes into L2 (its offsets were prefetched above)
                const int64_t ns0 = (int64_t)next * C::RS;
                const int64_t nend = P.n - ns0 < C::RS ? P.n : ns0 + C::RS;
                const int64_t a = align16_down((__ldg(P.off + ns0) + 7) & ~(int64_t)7);
                const int64_t b = align16_up(__ldg(P.off + nend));
                const int64_t bytes = b - a < (int64_t)C::PREFETCH ? b - a : (int64_t)C::PREFETCH;
                if (bytes > 0) bulk_prefetch_l2(P.base + a, (uint32_t)bytes);
            }
            first_fill = false;
            const bool ok = wait_copies(&S.bar, phase, &S.abort, P.status);
            phase ^= 1u;
            if (!ok) return;  // PMP_ETIMEOUT is in the device status word
            const uint32_t total = S.total, nmed = S.nmed;
            const uint32_t nwork = nmed + (total + 31) / 32;
            for (;;) {
                uint32_t w = 0;
                if (lane == 0) w = atomicAdd(&S.work, 1u);
                w = __shfl_sync(0xffffffffu, w, 0);
                if (w >= nwork) break;
                if (w < nmed) {
                    const int64_t i = s0 + (int64_t)S.rec[C::RS - 1 - w].x;
                    uint64_t st, len;
                    string_span(P.off, i, st, len);
                    range_medium<N>(P, S, i, P.base + st, len, b1);
                } else
                    range_group<N>(P, S, s0, 32 * (w - nmed), total, b1);
            }
            __syncthreads();
            x = y;
        }
        range = next;
    }
}

}  // namespace pm
