/*
 * pmo.h -- plain, slow, single-threaded CPU oracle for PM+ hashing
 * (Ivanchykhin, Ignatchenko, Lemire, "Regular and almost universal hashing:
 * an efficient implementation", arXiv 1609.09840).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline of the benchmark may load or call this code. The GPU library never
 * links, includes or calls it, and it shares no code with the GPU library.
 *
 * Every quantity is computed from its definition with exact multi-limb
 * integer arithmetic and a generic remainder (binary long division). The
 * paper's fast reduction (Sec. 6.2, Algorithm 2) is deliberately NOT used
 * here, so that the GPU path's reduction is checked against an independent
 * computation.
 */
#ifndef PMO_H
#define PMO_H
#include <stdint.h>
#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

/* Family parameters (Table "parameters", Sec. 6.1; primes from the table of
 * smallest primes above a power of two, Sec. 5). p = 2^n + k. */
typedef struct {
    int      n;      /* word width in bits: 8, 16, 32 or 64 */
    uint64_t k;      /* p = 2^n + k */
    uint64_t kappa;  /* keys a_i are drawn from (0, p - kappa) */
    int      m;      /* words per chunk (segment length of Algorithm 1) */
    int      L;      /* number of independent level functions f_1..f_L */
} pmo_params;

/* A value of [0, p): lo + 2^64 * hi, hi in {0,1}. For n <= 32 hi is 0. */
typedef struct { uint64_t lo, hi; } pmo_val;

enum { PMO_OK = 0, PMO_EINVAL = 1, PMO_ETOOLONG = 4 };

/* The two parameter sets of the paper (Table "parameters"). */
void pmo_params_pm32(pmo_params *out);
void pmo_params_pm64(pmo_params *out);

/* Number of key words: L * (1 + m), level-major, key[j*(1+m)] = b_{j+1},
 * key[j*(1+m) + i] = a_{j+1,i} (i = 1..m). */
size_t pmo_key_words(const pmo_params *P);

/* Key expansion from a seed (library convention, not fixed by the paper):
 * a splitmix64 stream started at `seed`; for each level j: b_j = top n bits
 * of the next draw, then for i = 1..m: draw until the top n bits lie in
 * [1, p - kappa - 1] (Definition of PM+-Multilinear, Sec. 5). */
int pmo_key_expand(const pmo_params *P, uint64_t seed, uint64_t *key);

/* splitmix64 output number `i` (0-based) of the stream started at `seed`. */
uint64_t pmo_splitmix64_at(uint64_t seed, uint64_t i);

/* Number of tree levels Algorithm 1 applies to a string of N0 padded words
 * (at least one level is always applied). 0 when N0 > m^L. */
int pmo_levels(const pmo_params *P, uint64_t n0);

/* Raw tree value h(s) in [0, p) of a byte string (Algorithm 1 with the byte
 * padding of Sec. 4: a 0x01 byte then zeros up to the word boundary). */
int pmo_tree_bytes(const pmo_params *P, const uint64_t *key,
                   const uint8_t *bytes, uint64_t len, pmo_val *out);

/* Same result computed with the bounded-memory streaming order described
 * at the end of Sec. 4 (at most m values kept per level). */
int pmo_tree_bytes_streaming(const pmo_params *P, const uint64_t *key,
                             const uint8_t *bytes, uint64_t len, pmo_val *out);

/* Algorithm 1 on a string of N words s_1..s_N (each < 2^n): the value 1 is
 * appended, then the level loop runs. Used for the worked example of Fig. 1. */
int pmo_tree_words(const pmo_params *P, const uint64_t *key,
                   const uint64_t *words, uint64_t N, pmo_val *out);

/* One chunk function f(s) = (b + sum_i a_i s_i) mod p (eq. 2wlinear), with
 * b = fkey[0] and a_i = fkey[i]; s holds m values of [0, p). */
pmo_val pmo_chunk(const pmo_params *P, const uint64_t *fkey, const pmo_val *s);

/* Output step (Sec. 5 end, Sec. 7): z = h mod 2^n, then the bit mixer (for
 * n = 32 and n = 64; for the toy widths the mixer is the identity). */
uint64_t pmo_output(const pmo_params *P, pmo_val h);
uint32_t pmo_mix32(uint32_t z);
uint64_t pmo_mix64(uint64_t z);

/* Full hash of one byte string: output(tree_bytes(.)). */
int pmo_hash_bytes(const pmo_params *P, const uint64_t *key,
                   const uint8_t *bytes, uint64_t len, uint64_t *out);

/* Batch of strings packed in one buffer: string i occupies bytes
 * [align8(offsets[i]), offsets[i+1]) of `base`. raw != 0 stores the tree
 * value's low 64 bits and high bit into out[2i], out[2i+1]; raw == 0 stores
 * the hash into out[i]. Returns the first error. */
int pmo_hash_batch(const pmo_params *P, const uint64_t *key,
                   const uint8_t *base, const int64_t *offsets, int64_t n,
                   int raw, uint64_t *out);

/* Generic remainder of a little-endian multi-limb number (nlimbs 32-bit
 * limbs, nlimbs <= 8) by p = 2^n + k: exposed so that the tests can pin it
 * against Python's arbitrary-precision '%'. */
pmo_val pmo_mod_limbs(const pmo_params *P, const uint32_t *limbs, int nlimbs);

#ifdef __cplusplus
}
#endif
#endif
