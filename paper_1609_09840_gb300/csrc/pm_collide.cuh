// pm_collide.cuh -- collision counting over many keys (property tests).
//
// Sec. 3 (Lemma 1, after Dai and Krovetz) and the universality lemma of
// Sec. 5: PM+-Multilinear is 1/(p - 1 - kappa)-almost Delta-universal, so
// its values reduced mod 2^t collide for two distinct strings with
// probability at most ceil((2p - 1) / 2^t) / (p - 1 - kappa) over the key.
// k_collide measures that probability: thread q takes the key of seed
// seed0 + q (the key convention of k_keygen: b_1 = the top n bits of draw 0,
// then a_{1,i} = the top n bits of the next draw, redrawn until in
// [1, p - kappa - 1]), hashes two one-chunk strings A and B with it (the raw
// value h in [0, p) of eq. 2wlinear, Sec. 6.2, Alg. 2) and counts the keys
// for which the low t bits of h(A) and h(B) agree. Only the key words the
// strings need are drawn, so 10^8 keys take a fraction of a second.
#pragma once
#include "pm_kernels.cuh"

namespace pm {

constexpr int COLLIDE_MAX_WORDS = 16;  // words of the padded strings (one chunk)

template <int N>
__global__ void __launch_bounds__(256) k_collide(uint64_t seed0, uint64_t nkeys, const uint8_t *a, uint32_t len_a,
                                                 const uint8_t *b, uint32_t len_b, int t,
                                                 unsigned long long *count) {
    typedef typename Fam<N>::word word;
    constexpr uint64_t W = Fam<N>::W;
    const uint64_t wmax = N == 64 ? ~0ull : ((1ull << N) - 1);
    const uint64_t amax = wmax - (Fam<N>::KAPPA - Fam<N>::K);  // p - kappa - 1
    const int na = (int)(len_a / W) + 1, nb = (int)(len_b / W) + 1;
    const int nw = na > nb ? na : nb;
    // the padded words of both strings (Sec. 4: bytes, then 0x01, then zeros)
    word sa[COLLIDE_MAX_WORDS], sb[COLLIDE_MAX_WORDS];
#pragma unroll
    for (int i = 0; i < COLLIDE_MAX_WORDS; ++i) {
        const uint64_t ua = load_unit_padded(a, len_a, (uint64_t)(i * W / 8));
        const uint64_t ub = load_unit_padded(b, len_b, (uint64_t)(i * W / 8));
        if constexpr (N == 32) {
            sa[i] = (word)((i & 1) ? ua >> 32 : ua);
            sb[i] = (word)((i & 1) ? ub >> 32 : ub);
        } else {
            sa[i] = ua;
            sb[i] = ub;
        }
    }
    const uint64_t tmask = t >= 64 ? ~0ull : ((1ull << t) - 1);
    unsigned long long hits = 0;
    const uint64_t stride = (uint64_t)gridDim.x * blockDim.x;
    for (uint64_t q = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; q < nkeys; q += stride) {
        const uint64_t seed = seed0 + q;
        uint64_t draw = 0;
        const uint64_t bb = splitmix64_at(seed, draw++) >> (64 - N);
        U192 ha = {bb, 0, 0}, hb = {bb, 0, 0};
        for (int i = 0; i < nw; ++i) {
            uint64_t ai;
            do {
                ai = splitmix64_at(seed, draw++) >> (64 - N);
            } while (ai < 1 || ai > amax);
            Val x;
            x.hi = 0;
            if (i < na) {
                x.lo = (uint64_t)sa[i];
                mac(ha, (word)ai, x);
            }
            if (i < nb) {
                x.lo = (uint64_t)sb[i];
                mac(hb, (word)ai, x);
            }
        }
        const Val va = reduce<N>(ha), vb = reduce<N>(hb);
        hits += ((va.lo ^ vb.lo) & tmask) == 0;
    }
    // warp-aggregated count
#pragma unroll
    for (int d = 16; d > 0; d >>= 1) hits += __shfl_down_sync(0xffffffffu, hits, d);
    if ((threadIdx.x & 31) == 0 && hits) atomicAdd(count, hits);
}

}  // namespace pm
