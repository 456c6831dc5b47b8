/*
 * pmo.c -- plain, slow, single-threaded CPU oracle for PM+ hashing
 * (arXiv 1609.09840).
 *
 * TEST INFRASTRUCTURE. Only the test suite, the smoke check and the CPU
 * baseline of the benchmark may load or call this code; the GPU library
 * shares nothing with it.
 *
 * Passages followed:
 *   - Definition of PM+-Multilinear, eq. (2wlinear), Sec. 5:
 *       f(s) = (b + sum_{i=1}^m a_i s_i) mod p, b in [0,2^n), a_i in (0,p-kappa).
 *   - Table "parameters" (Sec. 6.1): p = 2^32+15, kappa = 28 and
 *     p = 2^64+13, kappa = 24; m = 128; L = 8.
 *   - Algorithm 1 (tree-based algorithm, Sec. 4): append 1, then repeatedly
 *     zero-pad to a multiple of m and replace the string by the values of f_j
 *     on its m-segments, j = 1, 2, ..., until one value remains. At least one
 *     level is always applied (Sec. 4: "If L=1 simply return f_1(sigma)"
 *     padded to length m; Fig. 1a hashes the one-chunk string "ab").
 *   - Byte strings (Sec. 4, last paragraph): the appended 1 is a 0x01 byte
 *     followed by zeros up to the machine-word boundary; words are taken in
 *     little-endian byte order (the paper's x86/ARM targets).
 *   - Bounded-memory streaming order (Sec. 4): same result with at most m
 *     values kept per level.
 *   - Output step (Sec. 5 end): h mod 2^n; mixer (Sec. 7) for n = 32, 64.
 *
 * Arithmetic: exact multi-limb integers (32-bit limbs) and the remainder by
 * binary long division. The paper's reduction shortcut (Sec. 6.2,
 * Algorithm 2) is not used.
 */
#include "pmo.h"
#include <stdlib.h>
#include <string.h>

/* ------------------------------------------------------------------------ */
/* Multi-limb unsigned integers: 8 little-endian 32-bit limbs (256 bits).    */
/* The largest number formed is S < 2^n + m * 2^(2n+1) <= 2^140 for n = 64.  */
/* ------------------------------------------------------------------------ */
#define NL 8
typedef struct { uint32_t d[NL]; } big;

static void big_zero(big *x) { memset(x, 0, sizeof *x); }

static void big_from_val(big *x, pmo_val v) {
    big_zero(x);
    x->d[0] = (uint32_t)v.lo;
    x->d[1] = (uint32_t)(v.lo >> 32);
    x->d[2] = (uint32_t)v.hi;
    x->d[3] = (uint32_t)(v.hi >> 32);
}

static void big_from_u64(big *x, uint64_t v) {
    pmo_val t;
    t.lo = v;
    t.hi = 0;
    big_from_val(x, t);
}

static pmo_val big_to_val(const big *x) {
    pmo_val v;
    v.lo = (uint64_t)x->d[0] | ((uint64_t)x->d[1] << 32);
    v.hi = (uint64_t)x->d[2] | ((uint64_t)x->d[3] << 32);
    return v;
}

/* acc += x */
static void big_add(big *acc, const big *x) {
    uint64_t carry = 0;
    for (int i = 0; i < NL; ++i) {
        uint64_t t = (uint64_t)acc->d[i] + x->d[i] + carry;
        acc->d[i] = (uint32_t)t;
        carry = t >> 32;
    }
}

/* acc -= x, requires acc >= x */
static void big_sub(big *acc, const big *x) {
    uint64_t borrow = 0;
    for (int i = 0; i < NL; ++i) {
        uint64_t t = (uint64_t)acc->d[i] - x->d[i] - borrow;
        acc->d[i] = (uint32_t)t;
        borrow = (t >> 32) & 1;
    }
}

static int big_cmp(const big *a, const big *b) {
    for (int i = NL - 1; i >= 0; --i) {
        if (a->d[i] != b->d[i]) return a->d[i] < b->d[i] ? -1 : 1;
    }
    return 0;
}

/* acc += x * y (schoolbook product) */
static void big_mul_add(big *acc, const big *x, const big *y) {
    big prod;
    big_zero(&prod);
    for (int i = 0; i < NL; ++i) {
        uint64_t carry = 0;
        if (x->d[i] == 0) continue;
        for (int j = 0; i + j < NL; ++j) {
            uint64_t t = (uint64_t)x->d[i] * y->d[j] + prod.d[i + j] + carry;
            prod.d[i + j] = (uint32_t)t;
            carry = t >> 32;
        }
    }
    big_add(acc, &prod);
}

static int big_bit(const big *x, int i) { return (int)((x->d[i / 32] >> (i % 32)) & 1u); }

static void big_shl1(big *x) {
    for (int i = NL - 1; i > 0; --i) x->d[i] = (x->d[i] << 1) | (x->d[i - 1] >> 31);
    x->d[0] <<= 1;
}

/* r = x mod p, by binary long division (remainder only). */
static void big_mod(big *r, const big *x, const big *p) {
    int top = NL * 32 - 1;
    big_zero(r);
    while (top >= 0 && !big_bit(x, top)) --top;
    for (int i = top; i >= 0; --i) {
        big_shl1(r);
        r->d[0] |= (uint32_t)big_bit(x, i);
        if (big_cmp(r, p) >= 0) big_sub(r, p);
    }
}

/* p = 2^n + k */
static void big_prime(big *p, const pmo_params *P) {
    big kk;
    big_zero(p);
    p->d[P->n / 32] |= 1u << (P->n % 32);
    big_from_u64(&kk, P->k);
    big_add(p, &kk);
}

/* ------------------------------------------------------------------------ */
/* Parameters                                                               */
/* ------------------------------------------------------------------------ */
void pmo_params_pm32(pmo_params *out) {
    out->n = 32;
    out->k = 15;
    out->kappa = 28;
    out->m = 128;
    out->L = 8;
}

void pmo_params_pm64(pmo_params *out) {
    out->n = 64;
    out->k = 13;
    out->kappa = 24;
    out->m = 128;
    out->L = 8;
}

static int params_ok(const pmo_params *P) {
    if (!P) return 0;
    if (P->n != 8 && P->n != 16 && P->n != 32 && P->n != 64) return 0;
    if (P->m < 2 || P->m > 4096 || P->L < 1 || P->L > 64) return 0;
    return 1;
}

size_t pmo_key_words(const pmo_params *P) { return (size_t)P->L * (size_t)(1 + P->m); }

/* ------------------------------------------------------------------------ */
/* Key expansion (library convention; the paper fixes only the ranges).      */
/* splitmix64 (Steele, Lea, Flood 2014): state advances by the golden-gamma  */
/* constant, and each state is passed through the mix64 finaliser.           */
/* ------------------------------------------------------------------------ */
static uint64_t splitmix64_mix(uint64_t z) {
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ULL;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebULL;
    return z ^ (z >> 31);
}

uint64_t pmo_splitmix64_at(uint64_t seed, uint64_t i) {
    return splitmix64_mix(seed + (i + 1) * 0x9e3779b97f4a7c15ULL);
}

static uint64_t top_bits(uint64_t x, int n) { return n == 64 ? x : (x >> (64 - n)); }

/* a is acceptable iff 1 <= a <= p - kappa - 1 = (2^n - 1) - (kappa - k). */
static int key_in_range(const pmo_params *P, uint64_t a) {
    uint64_t wmax = P->n == 64 ? ~0ULL : ((1ULL << P->n) - 1);
    if (a < 1) return 0;
    if (P->kappa >= P->k) return a <= wmax - (P->kappa - P->k);
    return 1; /* p - kappa - 1 >= 2^n: every non-zero n-bit value is allowed */
}

int pmo_key_expand(const pmo_params *P, uint64_t seed, uint64_t *key) {
    uint64_t draw = 0;
    if (!params_ok(P) || !key) return PMO_EINVAL;
    for (int j = 0; j < P->L; ++j) {
        uint64_t *f = key + (size_t)j * (size_t)(1 + P->m);
        f[0] = top_bits(pmo_splitmix64_at(seed, draw++), P->n); /* b_j in [0, 2^n) */
        for (int i = 1; i <= P->m; ++i) {
            uint64_t a;
            do {
                a = top_bits(pmo_splitmix64_at(seed, draw++), P->n);
            } while (!key_in_range(P, a));
            f[i] = a;
        }
    }
    return PMO_OK;
}

/* ------------------------------------------------------------------------ */
/* Tree construction                                                        */
/* ------------------------------------------------------------------------ */
int pmo_levels(const pmo_params *P, uint64_t n0) {
    int lv = 0;
    uint64_t N = n0;
    if (!params_ok(P) || n0 == 0) return 0;
    do {
        N = (N + (uint64_t)P->m - 1) / (uint64_t)P->m;
        ++lv;
    } while (N > 1);
    return lv <= P->L ? lv : 0;
}

/* f(s) = (b + sum_{i=1}^m a_i s_i) mod p with b = fkey[0], a_i = fkey[i]. */
pmo_val pmo_chunk(const pmo_params *P, const uint64_t *fkey, const pmo_val *s) {
    big S, a, x, p, r;
    big_from_u64(&S, fkey[0]);
    for (int i = 1; i <= P->m; ++i) {
        big_from_u64(&a, fkey[i]);
        big_from_val(&x, s[i - 1]);
        big_mul_add(&S, &a, &x);
    }
    big_prime(&p, P);
    big_mod(&r, &S, &p);
    return big_to_val(&r);
}

/* Source of the level-1 string sigma. */
typedef struct {
    const uint8_t  *bytes;  /* byte mode */
    uint64_t        len;
    const uint64_t *words;  /* word mode: s_1..s_N, then the appended 1 */
    uint64_t        N;
    int             word_mode;
} sigma_src;

/* Word i (0-based) of sigma. Byte mode: little-endian bytes of the string,
 * the 0x01 pad byte at position len, zeros after it. */
static uint64_t sigma_word(const pmo_params *P, const sigma_src *src, uint64_t i) {
    if (src->word_mode) return i < src->N ? src->words[i] : (i == src->N ? 1u : 0u);
    {
        int W = P->n / 8;
        uint64_t w = 0;
        for (int b = 0; b < W; ++b) {
            uint64_t pos = i * (uint64_t)W + (uint64_t)b;
            uint64_t byte = pos < src->len ? src->bytes[pos] : (pos == src->len ? 1u : 0u);
            w |= byte << (8 * b);
        }
        return w;
    }
}

static uint64_t sigma_len(const pmo_params *P, const sigma_src *src) {
    return src->word_mode ? src->N + 1 : src->len / (uint64_t)(P->n / 8) + 1;
}

static const uint64_t *level_key(const pmo_params *P, const uint64_t *key, int j /* 1-based */) {
    return key + (size_t)(j - 1) * (size_t)(1 + P->m);
}

/* Algorithm 1, level by level. */
static int tree_levelwise(const pmo_params *P, const uint64_t *key, const sigma_src *src,
                          pmo_val *out) {
    uint64_t n0 = sigma_len(P, src), count, c;
    uint64_t m = (uint64_t)P->m;
    pmo_val *vals, *seg;
    int j = 1;
    if (pmo_levels(P, n0) == 0) return PMO_ETOOLONG;
    seg = (pmo_val *)malloc(sizeof(pmo_val) * m);
    count = (n0 + m - 1) / m;
    vals = (pmo_val *)malloc(sizeof(pmo_val) * count);
    if (!seg || !vals) {
        free(seg);
        free(vals);
        return PMO_EINVAL;
    }
    /* level 1: zero-pad sigma to a multiple of m, apply f_1 to each segment */
    for (c = 0; c < count; ++c) {
        for (uint64_t i = 0; i < m; ++i) {
            uint64_t idx = c * m + i;
            seg[i].lo = idx < n0 ? sigma_word(P, src, idx) : 0;
            seg[i].hi = 0;
        }
        vals[c] = pmo_chunk(P, level_key(P, key, 1), seg);
    }
    /* while sigma has more than one value: next level */
    while (count > 1) {
        uint64_t ncount = (count + m - 1) / m;
        pmo_val *next = (pmo_val *)malloc(sizeof(pmo_val) * ncount);
        ++j;
        if (!next || j > P->L) {
            free(next);
            free(vals);
            free(seg);
            return PMO_ETOOLONG;
        }
        for (c = 0; c < ncount; ++c) {
            for (uint64_t i = 0; i < m; ++i) {
                uint64_t idx = c * m + i;
                if (idx < count) {
                    seg[i] = vals[idx];
                } else {
                    seg[i].lo = 0;
                    seg[i].hi = 0;
                }
            }
            next[c] = pmo_chunk(P, level_key(P, key, j), seg);
        }
        free(vals);
        vals = next;
        count = ncount;
    }
    *out = vals[0];
    free(vals);
    free(seg);
    return PMO_OK;
}

/* Bounded-memory order (Sec. 4): each finished chunk value is pushed to the
 * next level's buffer; a full buffer is hashed and pushed further up. */
typedef struct {
    const pmo_params *P;
    const uint64_t   *key;
    pmo_val          *buf;   /* L+1 rows of m values; row j is level j's input */
    uint64_t         *fill;  /* values currently buffered per level */
    uint64_t         *total; /* values ever pushed per level */
    int               err;
} stream_state;

static void stream_push(stream_state *st, int j, pmo_val v) {
    uint64_t m = (uint64_t)st->P->m;
    /* level j holds inputs of f_j; level L+1 may only receive the final value */
    if (j > st->P->L + 1 || (j == st->P->L + 1 && st->total[j] > 0)) {
        st->err = PMO_ETOOLONG;
        return;
    }
    st->buf[(size_t)j * m + st->fill[j]] = v;
    st->fill[j]++;
    st->total[j]++;
    if (st->fill[j] == m) {
        pmo_val r = pmo_chunk(st->P, level_key(st->P, st->key, j), st->buf + (size_t)j * m);
        st->fill[j] = 0;
        stream_push(st, j + 1, r);
    }
}

static int tree_streaming(const pmo_params *P, const uint64_t *key, const sigma_src *src,
                          pmo_val *out) {
    uint64_t n0 = sigma_len(P, src), m = (uint64_t)P->m, nchunks, c;
    stream_state st;
    pmo_val *seg;
    int j, rc = PMO_OK;
    if (pmo_levels(P, n0) == 0) return PMO_ETOOLONG;
    st.P = P;
    st.key = key;
    st.err = PMO_OK;
    st.buf = (pmo_val *)calloc((size_t)(P->L + 2) * m, sizeof(pmo_val));
    st.fill = (uint64_t *)calloc((size_t)P->L + 2, sizeof(uint64_t));
    st.total = (uint64_t *)calloc((size_t)P->L + 2, sizeof(uint64_t));
    seg = (pmo_val *)malloc(sizeof(pmo_val) * m);
    if (!st.buf || !st.fill || !st.total || !seg) {
        rc = PMO_EINVAL;
        goto done;
    }
    /* level 1 chunks, pushed into level 2 as they complete */
    nchunks = (n0 + m - 1) / m;
    for (c = 0; c < nchunks; ++c) {
        for (uint64_t i = 0; i < m; ++i) {
            uint64_t idx = c * m + i;
            seg[i].lo = idx < n0 ? sigma_word(P, src, idx) : 0;
            seg[i].hi = 0;
        }
        stream_push(&st, 2, pmo_chunk(P, level_key(P, key, 1), seg));
        if (st.err) break;
    }
    /* completion: level j received total[j] values; one value ends the tree,
     * otherwise the partial buffer (if any) is zero-padded and hashed. */
    for (j = 2; !st.err; ++j) {
        if (j > P->L + 1) {
            st.err = PMO_ETOOLONG;
            break;
        }
        if (st.total[j] == 1) {
            *out = st.buf[(size_t)j * m];
            break;
        }
        if (st.fill[j] > 0) {
            if (j > P->L) {
                st.err = PMO_ETOOLONG;
                break;
            }
            pmo_val *row = st.buf + (size_t)j * m;
            pmo_val r;
            for (uint64_t i = st.fill[j]; i < m; ++i) {
                row[i].lo = 0;
                row[i].hi = 0;
            }
            r = pmo_chunk(P, level_key(P, key, j), row);
            st.fill[j] = 0;
            stream_push(&st, j + 1, r);
        }
    }
    rc = st.err;
done:
    free(st.buf);
    free(st.fill);
    free(st.total);
    free(seg);
    return rc;
}

int pmo_tree_bytes(const pmo_params *P, const uint64_t *key, const uint8_t *bytes, uint64_t len,
                   pmo_val *out) {
    sigma_src src;
    if (!params_ok(P) || !key || !out || (!bytes && len)) return PMO_EINVAL;
    memset(&src, 0, sizeof src);
    src.bytes = bytes;
    src.len = len;
    return tree_levelwise(P, key, &src, out);
}

int pmo_tree_bytes_streaming(const pmo_params *P, const uint64_t *key, const uint8_t *bytes,
                             uint64_t len, pmo_val *out) {
    sigma_src src;
    if (!params_ok(P) || !key || !out || (!bytes && len)) return PMO_EINVAL;
    memset(&src, 0, sizeof src);
    src.bytes = bytes;
    src.len = len;
    return tree_streaming(P, key, &src, out);
}

int pmo_tree_words(const pmo_params *P, const uint64_t *key, const uint64_t *words, uint64_t N,
                   pmo_val *out) {
    sigma_src src;
    if (!params_ok(P) || !key || !out || (!words && N)) return PMO_EINVAL;
    memset(&src, 0, sizeof src);
    src.words = words;
    src.N = N;
    src.word_mode = 1;
    return tree_levelwise(P, key, &src, out);
}

/* ------------------------------------------------------------------------ */
/* Output step                                                              */
/* ------------------------------------------------------------------------ */
uint32_t pmo_mix32(uint32_t z) { /* Sec. 7, 32-bit mixer */
    z = z ^ (z >> 13);
    z = z * 0xab3be54fu;
    z = z ^ (z >> 16);
    return z;
}

uint64_t pmo_mix64(uint64_t z) { /* Sec. 7, 64-bit mixer */
    z = z ^ (z >> 33);
    z = z * 0xc4ceb9fe1a85ec53ULL;
    z = z ^ (z >> 33);
    return z;
}

uint64_t pmo_output(const pmo_params *P, pmo_val h) {
    uint64_t z = P->n == 64 ? h.lo : (h.lo & ((1ULL << P->n) - 1)); /* h mod 2^n */
    if (P->n == 64) return pmo_mix64(z);
    if (P->n == 32) return pmo_mix32((uint32_t)z);
    return z;
}

int pmo_hash_bytes(const pmo_params *P, const uint64_t *key, const uint8_t *bytes, uint64_t len,
                   uint64_t *out) {
    pmo_val h;
    int rc = pmo_tree_bytes(P, key, bytes, len, &h);
    if (rc == PMO_OK) *out = pmo_output(P, h);
    return rc;
}

int pmo_hash_batch(const pmo_params *P, const uint64_t *key, const uint8_t *base,
                   const int64_t *offsets, int64_t n, int raw, uint64_t *out) {
    if (!params_ok(P) || !key || !offsets || !out || n < 0) return PMO_EINVAL;
    for (int64_t i = 0; i < n; ++i) {
        int64_t start = (offsets[i] + 7) & ~(int64_t)7, end = offsets[i + 1];
        pmo_val h;
        int rc;
        if (offsets[i] < 0 || end < start) return PMO_EINVAL;
        rc = pmo_tree_bytes(P, key, base + start, (uint64_t)(end - start), &h);
        if (rc != PMO_OK) return rc;
        if (raw) {
            out[2 * i] = h.lo;
            out[2 * i + 1] = h.hi;
        } else {
            out[i] = pmo_output(P, h);
        }
    }
    return PMO_OK;
}

pmo_val pmo_mod_limbs(const pmo_params *P, const uint32_t *limbs, int nlimbs) {
    big x, p, r;
    big_zero(&x);
    for (int i = 0; i < nlimbs && i < NL; ++i) x.d[i] = limbs[i];
    big_prime(&p, P);
    big_mod(&r, &x, &p);
    return big_to_val(&r);
}
