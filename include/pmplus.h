/*
 * pmplus.h -- C ABI of the GB300 (sm_103a) PM+ hashing library.
 *
 * PM+ (Ivanchykhin, Ignatchenko, Lemire, "Regular and almost universal
 * hashing: an efficient implementation", arXiv 1609.09840) hashes a byte
 * string s with L = 8 independent PM+-Multilinear functions
 *     f_j(s_1..s_m) = (b_j + sum_{i=1}^m a_{j,i} s_i) mod p     (Sec. 5, eq. 2wlinear)
 * over words of n = 32 or 64 bits, p = 2^32+15 or 2^64+13, m = 128
 * (Table "parameters", Sec. 6.1), applied level by level in the tree of
 * Algorithm 1 (Sec. 4) to the string padded with a 0x01 byte and zeros up to
 * the word boundary (Sec. 4, last paragraph; words are little-endian). The
 * output is the mixer of Sec. 7 applied to h(s) mod 2^n (Sec. 5, end).
 *
 * General rules for every entry point:
 *  - Pointers prefixed d_ are device pointers on the current CUDA device;
 *    pointers prefixed host_ are host pointers.
 *  - `stream` is a cudaStream_t (passed as void*); NULL means the legacy
 *    default stream. Every hashing call is asynchronous on that stream and
 *    never synchronizes, allocates or frees memory (object creation and
 *    destruction -- keys, streams, graphs, servers -- may).
 *  - Every call returns a pmp_status. Argument errors are reported
 *    synchronously and nothing is launched. A kernel launch failure returns
 *    PMP_ECUDA. Errors detected on the device (a bounded wait that ran out)
 *    are recorded in a device status word read by pmp_device_status().
 *  - The caller owns all d_ buffers and keeps them alive until the work on
 *    `stream` is done. The library owns the key object and its device copy.
 *  - Scratch memory: calls that need device scratch take (d_scratch,
 *    scratch_bytes); the required size comes from the matching *_scratch_bytes
 *    query. Scratch is caller-owned, must not be shared by calls that may run
 *    concurrently, and needs no initialisation.
 */
#ifndef PMPLUS_H
#define PMPLUS_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
    PMP_OK = 0,
    PMP_EINVAL = 1,   /* bad argument (null pointer, wrong key width, bad size) */
    PMP_ENOMEM = 2,   /* device allocation failed (pmp_key_create, pmp_stream_create) */
    PMP_ECUDA = 3,    /* a CUDA runtime call or kernel launch failed */
    PMP_ETOOLONG = 4, /* string longer than m^L - 1 words: more than 8 levels */
    PMP_ETIMEOUT = 5, /* a bounded device-side wait ran out (device status) */
    PMP_EALIGN = 6,   /* a pointer lacks the documented alignment */
    PMP_ESCRATCH = 7  /* input needs more scratch than given (or than pmp_hash64_noalloc's fixed buffer) */
} pmp_status;

typedef struct pmp_key pmp_key; /* opaque */

/* ---------------------------------------------------------------------------
 * Keys (Sec. 5 Definition; Algorithm 1 requires L independent functions).
 * Layout (library convention; the paper fixes only the ranges): level-major,
 * L = 8 rows of 1 + m = 129 words: row j holds b_{j+1} then a_{j+1,1..128},
 * as uint32 words for width 32 and uint64 words for width 64.
 * Generation: the splitmix64 stream (Steele, Lea, Flood 2014) started at
 * `seed` -- output i is mix64(seed + (i+1) * 0x9e3779b97f4a7c15). For each
 * level: b = top n bits of the next output; then each a_i = top n bits of
 * the next output, redrawn until it lies in [1, p - kappa - 1]
 * (kappa = 28 for width 32, 24 for width 64, Table "parameters").
 * ------------------------------------------------------------------------- */

/* Create a key of `width` 32 or 64 bits on the current device. The key is
 * expanded by a device kernel; the call synchronizes once. *out receives the
 * key (free with pmp_key_destroy). Errors: PMP_EINVAL (width, out == NULL),
 * PMP_ENOMEM, PMP_ECUDA. */
int pmp_key_create(uint64_t seed, int width, pmp_key **out);

/* Copy the key words (level-major, as above) to host memory. cap_bytes must
 * be >= 8*129*(width/8). Synchronous. */
int pmp_key_export(const pmp_key *key, void *host_dst, size_t cap_bytes);

/* Width (32 or 64) of a key, 0 for NULL. */
int pmp_key_width(const pmp_key *key);

/* Free a key (synchronizes with the device first). NULL is ignored. */
void pmp_key_destroy(pmp_key *key);

/* ---------------------------------------------------------------------------
 * One buffer: out = mix(h(buf[0..len)) mod 2^n) (Algorithm 1 over all levels,
 * Sec. 5 output step, Sec. 7 mixer).
 * d_buf: len bytes, 16-byte aligned (PMP_EALIGN otherwise); may be NULL iff
 *        len == 0.
 * d_out: one uint32 (pmp_hash32) or uint64 (pmp_hash64).
 * Scratch: pmp_hash_scratch_bytes(width, len) bytes (level values of the
 *        tree levels >= 2 and their completion counters).
 * PMP_ETOOLONG when len >= 2^56 * (width/8).
 * ------------------------------------------------------------------------- */
size_t pmp_hash_scratch_bytes(int width, uint64_t len);
int pmp_hash32(const pmp_key *key, const void *d_buf, uint64_t len, uint32_t *d_out,
               void *d_scratch, size_t scratch_bytes, void *stream);
int pmp_hash64(const pmp_key *key, const void *d_buf, uint64_t len, uint64_t *d_out,
               void *d_scratch, size_t scratch_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * pmp_hash64 for callers that cannot allocate device memory. The paper has no
 * counterpart; this is a library convenience.
 *
 * Some callers may not call cudaMalloc at all: code that runs inside a host
 * application whose allocator owns every byte of device memory (an engine
 * plugin, a pre-partitioned serving process), and latency-critical paths
 * that cannot afford the implicit device synchronisation of an allocation.
 * They cannot provide the scratch that pmp_hash64 takes, so this entry point
 * uses a fixed scratch array compiled into the library instead: 1 MiB of
 * device memory per GPU that loads the library, held until the process exits.
 * It computes exactly what pmp_hash64 computes, with the same rules for
 * d_buf (16-byte aligned, len bytes), d_out (one uint64) and `stream`, and it
 * calls no allocating routine.
 *
 * Limit: inputs whose tree needs more than 1 MiB of level values and
 * counters -- about 8 GiB and longer -- return PMP_ESCRATCH; nothing is
 * launched. pmp_hash_noalloc_max_len() gives the exact bound.
 * The first call on each device looks up the array's device address (and
 * the per-device kernel settings); make that first call before any stream
 * capture on that device. The address is kept for the life of the process:
 * a device reset (cudaDeviceReset, or a rebuilt primary context) is not
 * supported afterwards -- the library's cached device state, this address
 * included, would be stale.
 * Every call on a device shares the one array and leaves its contents behind
 * (the counters that must start at zero are cleared by each call). Calls
 * whose work may overlap on the GPU -- on different streams, or from
 * different host threads -- race on the array and give wrong results:
 * serialise them, or use pmp_hash64 with separate scratch.
 * ------------------------------------------------------------------------- */
int pmp_hash64_noalloc(const pmp_key *key, const void *d_buf, uint64_t len, uint64_t *d_out,
                       void *stream);

/* Largest len pmp_hash64_noalloc accepts. */
uint64_t pmp_hash_noalloc_max_len(void);

/* ---------------------------------------------------------------------------
 * Ragged batch, one persistent launch sequence (the batched schedule).
 * d_base: packed strings, 8-byte aligned; string i occupies bytes
 *         [align8(d_offsets[i]), d_offsets[i+1]), so every string starts on
 *         an 8-byte boundary. The buffer must be readable up to
 *         align16(d_offsets[n]) (bytes are read with 16-byte copies and
 *         prefetched into L2 in 16-byte aligned ranges).
 * d_offsets: int64[n+1], non-decreasing after alignment (d_offsets[i+1] >=
 *         align8(d_offsets[i])), d_offsets[0] >= 0.
 * d_out:  n results (uint32 or uint64).
 * d_base must be 16-byte aligned (PMP_EALIGN otherwise).
 * Scratch: pmp_batch_scratch_bytes(width, n, data_bytes) bytes, with
 *         data_bytes >= d_offsets[n]: the work items of strings of at least
 *         32 level-1 chunks (one per level-2 chunk) and the tree storage of
 *         strings longer than m^2 words; the size depends on data_bytes only
 *         (n is checked, n >= 0, and otherwise unused). If the strings need
 *         more than the scratch covers, the device status reports
 *         PMP_ESCRATCH and some outputs are not written.
 * No string of a valid batch exceeds the L = 8 levels of the tree (m^L - 1
 * = 2^56 - 1 words): that would take 2^58 (32-bit) or 2^59 (64-bit) bytes of
 * device memory, so there is no PMP_ETOOLONG here; offsets that claim such a
 * string also break the readability rule above and are a caller error.
 * ------------------------------------------------------------------------- */
size_t pmp_batch_scratch_bytes(int width, int64_t n, uint64_t data_bytes);
int pmp_hash_batch32(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                     int64_t n, uint32_t *d_out, void *d_scratch, size_t scratch_bytes,
                     void *stream);
int pmp_hash_batch64(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                     int64_t n, uint64_t *d_out, void *d_scratch, size_t scratch_bytes,
                     void *stream);

/* pmp_hash_batch32/64 (the width is the key's; d_out holds n uint32 or
 * uint64) with a per-call device status word: d_status is one int in device
 * memory owned by the caller; a device-side error of this call (PMP_ESCRATCH,
 * PMP_ETIMEOUT) is written there if it still holds 0, besides the device
 * status word of pmp_device_status. Callers that run several batches at once
 * (the serving loop) use it to tell whose call failed; the caller zeroes it
 * before the call and reads it after the call's work completes. */
int pmp_hash_batch_status(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                          int64_t n, void *d_out, int *d_status, void *d_scratch,
                          size_t scratch_bytes, void *stream);

/* ---------------------------------------------------------------------------
 * Fixed-length keys (hash-table keys): n keys of len bytes each, key i at
 * d_keys + i * stride. Each key fits in one level-1 chunk (len < m W, i.e.
 * len < 512 bytes for 32-bit and < 1024 for 64-bit hashing), so its hash is
 * the chunk value of Sec. 5 (eq. 2wlinear, reduced by Sec. 6.2 and Alg. 2)
 * with the output step: the same value pmp_hash32/64 gives for the key
 * alone, and pmp_hash_batch32/64 gives for a batch of these strings, without
 * the offsets array (the keys' common length and stride replace it).
 * d_keys: 8-byte aligned (PMP_EALIGN otherwise); readable up to
 *   (n - 1) * stride + align8(len) bytes. stride: a multiple of 8 (PMP_EALIGN
 *   otherwise), >= len. len >= m W or stride < len: PMP_EINVAL.
 * d_out: n results (uint32 / uint64). Asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
int pmp_hash_fixed32(const pmp_key *key, const uint8_t *d_keys, int64_t n, uint32_t len, uint64_t stride,
                     uint32_t *d_out, void *stream);
int pmp_hash_fixed64(const pmp_key *key, const uint8_t *d_keys, int64_t n, uint32_t len, uint64_t stride,
                     uint64_t *d_out, void *stream);

/* ---------------------------------------------------------------------------
 * Collision counting over many keys (a property test of almost
 * Delta-universality; the paper has no such entry point). For the keys of
 * seeds seed0 .. seed0 + nkeys - 1 (the convention of pmp_key_create) it
 * adds to *d_count the number of keys for which the raw values (Sec. 5,
 * eq. 2wlinear, in [0, p)) of the one-chunk strings A and B agree in their
 * low t_bits bits. Sec. 3 (Lemma 1) and Sec. 5 bound that count's expected
 * value by nkeys * ceil((2p - 1) / 2^t) / (p - 1 - kappa) for A != B.
 * Strings: device bytes, 8-byte aligned (PMP_EALIGN), at most 16 words after
 * padding (len < 15 W + W: len <= 63 bytes for 32-bit, 127 for 64-bit;
 * PMP_EINVAL otherwise); read in 8-byte units. 1 <= t_bits <= width.
 * *d_count: a device counter the caller initialises; asynchronous.
 * ------------------------------------------------------------------------- */
int pmp_count_collisions(int width, uint64_t seed0, uint64_t nkeys, const uint8_t *d_a, uint32_t len_a,
                         const uint8_t *d_b, uint32_t len_b, int t_bits, unsigned long long *d_count,
                         void *stream);

/* ---------------------------------------------------------------------------
 * Toy members of the family, checked exhaustively (property tests; the paper
 * has no such entry point). Sec. 5's table of the smallest primes above
 * powers of two gives p = 2^8 + 1 and 2^16 + 1 (k = 1): with n = 8 or 16
 * every value of a word and every key of a short chunk can be enumerated.
 * n: 8 or 16 (words of n / 8 bytes, little-endian); 0 <= kappa < 2^n; key
 * words a in [1, p - kappa - 1]; 2 <= m <= 16; 1 <= L <= 8 (PMP_EINVAL
 * otherwise). Keys of seeds follow pmp_key_create's convention with these
 * parameters (b_j = the top n bits of a draw, a_{j,i} the top n bits of the
 * next draws redrawn until in range). Values are evaluated by the definition
 * (eq. 2wlinear with an exact remainder) and Algorithm 1's tree.
 *
 * pmp_toy_regularity: component-wise regularity (Sec. 3, Sec. 5). For each
 * key of seeds seed0 .. seed0 + nkeys - 1 and each word position c in
 * [comp0, comp0 + ncomp), word c of the len-byte string d_str (padded as in
 * Sec. 4) takes all 2^n values, each hashed through the whole tree (raw value
 * in [0, p)). d_counts[3 (q ncomp + c - comp0) + {0, 1, 2}] = the number of
 * raw values already seen, of values mod 2^n seen a second time, and of
 * values mod 2^n seen a third time or more: 0, <= k and 0 for a regular
 * family. d_raw: NULL, or nkeys * ncomp * 2^n uint32 receiving the raw values.
 * Positions must be whole string words (comp0 + ncomp <= len / W, else
 * PMP_EINVAL); len / W + 1 <= 128 words (PMP_EINVAL); the tree must end
 * within L levels (PMP_ETOOLONG); nkeys * ncomp < 2^31 (PMP_EINVAL).
 *
 * pmp_toy_delta_hist: almost Delta-universality (Sec. 5). s, t: host arrays
 * of m values in [0, p), s != t (PMP_EINVAL otherwise). d_hist: p counters
 * (uint64), overwritten: d_hist[e] = the number of keys (a_1 .. a_m) in
 * [1, p - kappa - 1]^m with f(s) - f(t) = e mod p (b cancels). The family is
 * 1 / (p - 1 - kappa)-almost Delta-universal: no count exceeds
 * (p - 1 - kappa)^(m - 1). At most 2^40 keys (PMP_EINVAL).
 * Both asynchronous on `stream`.
 * ------------------------------------------------------------------------- */
int pmp_toy_regularity(int n, int kappa, int m, int L, uint64_t seed0, uint32_t nkeys, const uint8_t *d_str,
                       uint32_t len, uint32_t comp0, uint32_t ncomp, uint32_t *d_counts, uint32_t *d_raw,
                       void *stream);
int pmp_toy_delta_hist(int n, int kappa, int m, const uint32_t *s, const uint32_t *t, unsigned long long *d_hist,
                       void *stream);

/* Raw tree values h(s) in [0, p) before the output step, for property tests
 * (regularity, universality): d_raw receives 2n uint64, (low 64 bits, high
 * bit) per string. Same layout rules and scratch as pmp_hash_batch{32,64}. */
int pmp_hash_batch_raw(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets,
                       int64_t n, uint64_t *d_raw, void *d_scratch, size_t scratch_bytes,
                       void *stream);

/* ---------------------------------------------------------------------------
 * Plain per-string path (comparison baseline): the same results as
 * pmp_hash_batch{32,64}, computed with one kernel launch per string. No
 * scratch. n launches are queued on `stream`.
 * ------------------------------------------------------------------------- */
int pmp_hash_batch32_plain(const pmp_key *key, const uint8_t *d_base,
                           const int64_t *d_offsets, int64_t n, uint32_t *d_out, void *stream);
int pmp_hash_batch64_plain(const pmp_key *key, const uint8_t *d_base,
                           const int64_t *d_offsets, int64_t n, uint64_t *d_out, void *stream);

/* ---------------------------------------------------------------------------
 * The device reduction of Sec. 6.2 (three-word sum -> two words, then
 * Algorithm 2), exposed for tests: d_S holds n triples (w0, w1, w2) of
 * uint64 giving S = w0 + 2^64 w1 + 2^128 w2 with S <= (2^n - 1) +
 * 128 (2^{2n} - 1); d_z receives n pairs (low 64 bits, high bit) of S mod p.
 * ------------------------------------------------------------------------- */
int pmp_debug_reduce(int width, const uint64_t *d_S, int64_t n, uint64_t *d_z, void *stream);

/* ---------------------------------------------------------------------------
 * Exhaustive checks of the 32-bit device arithmetic (property tests; the
 * paper has no such entry points). Each adds to *d_bad (a device counter the
 * caller initialises) the number of inputs that fail; asynchronous.
 * pmp_check_alg2_32: Algorithm 2 as read for this library (Sec. 6.2: input
 *   v0 + 2^32 v1 with v1 <= 2) on every v0 < 2^32 and v1 in {0, 1, 2},
 *   against (v0 + 2^32 v1) mod p by the integer remainder (p = 2^32 + 15).
 * pmp_check_reduce32: the device reduction of S = r0 + 2^32 r1[j] +
 *   2^64 r2[j] on every r0 < 2^32, for each of npairs (1..32) host pairs
 *   with r2[j] <= 128 (the three-word sums of Sec. 6.2), against S mod p
 *   by the integer remainder (PMP_EINVAL otherwise).
 * pmp_check_mix32: the 32-bit mixer of Sec. 7 followed by its inverse on
 *   every input; a_inv: the inverse of the mixer's odd multiplier mod 2^32.
 *   No failure means the mixer is a bijection.
 * ------------------------------------------------------------------------- */
int pmp_check_alg2_32(unsigned long long *d_bad, void *stream);
int pmp_check_reduce32(const uint32_t *r1, const uint32_t *r2, int npairs, unsigned long long *d_bad,
                       void *stream);
int pmp_check_mix32(uint32_t a_inv, unsigned long long *d_bad, void *stream);

/* ---------------------------------------------------------------------------
 * Failure-path test of the bounded device waits: one warp waits on an
 * mbarrier phase that never completes. The wait gives up after its limit
 * (2 s), records PMP_ETIMEOUT in the device status word (read and cleared by
 * pmp_device_status) and the kernel returns; the context stays usable.
 * *d_result (device int) = 1 if the wait reported success, else 0.
 * ------------------------------------------------------------------------- */
int pmp_debug_wait_timeout(int *d_result, void *stream);

/* ---------------------------------------------------------------------------
 * CUDA graphs of one call (library convenience). pmp_graph_hash /
 * pmp_graph_batch capture the launches of pmp_hash{32,64} /
 * pmp_hash_batch{32,64} (chosen by the key's width) with exactly these
 * arguments into an executable graph; pmp_graph_launch replays it on
 * `stream`, recomputing the hash of whatever the buffers hold then. The
 * arguments' buffers must stay valid while the graph exists; the tuning
 * knobs in effect at capture time are frozen into it.
 * ------------------------------------------------------------------------- */
typedef struct pmp_graph pmp_graph;
int pmp_graph_hash(const pmp_key *key, const void *d_buf, uint64_t len, void *d_out,
                   void *d_scratch, size_t scratch_bytes, pmp_graph **out);
int pmp_graph_batch(const pmp_key *key, const uint8_t *d_base, const int64_t *d_offsets, int64_t n,
                    void *d_out, void *d_scratch, size_t scratch_bytes, pmp_graph **out);
int pmp_graph_launch(pmp_graph *g, void *stream);
void pmp_graph_destroy(pmp_graph *g);

/* ---------------------------------------------------------------------------
 * Serving loop (a library runtime; the paper has no counterpart). One
 * scheduler thread per server admits hash requests in arrival order as soon
 * as one of `slots` CUDA streams is idle and the request's device memory fits
 * in a device arena of `budget_bytes` (allocated once by pmp_server_create),
 * so requests that arrive while others are running start at once and
 * overlap on the device (continuous batching). A request is either a packed
 * batch, copied to the device, hashed with pmp_hash_batch_status using the
 * server's resident keys and copied back, or a piece of a string held by the
 * server (a pmp_stream whose partial tree state stays on the device between
 * requests; Sec. 4's bounded-memory order). A request is done when its
 * results are visible in host memory. The scheduler issues copies and
 * launches without holding the lock that submit/wait take.
 *
 * Host buffers should be page-locked (cudaHostAlloc or cudaHostRegister):
 * copies from pageable memory are staged by the driver and serialize the
 * requests (results are the same).
 *
 * pmp_server_create: key32/key64 stay owned by the caller and must outlive
 *   the server. PMP_ENOMEM if the arena cannot be allocated.
 * pmp_server_submit: a packed batch in HOST memory (layout of
 *   pmp_hash_batch32/64); host_out receives n results of `width` bits. The
 *   buffers must stay valid and untouched until the request is done.
 *   Returns a ticket; PMP_ENOMEM if the request alone needs more than the
 *   budget.
 * pmp_server_stream_open: a string of `width`-bit hashing held by the server
 *   (its device state allocated now, on the server's device); *stream_id
 *   names it.
 * pmp_server_submit_piece: appends `len` bytes from host memory to string
 *   `stream_id` (a request of its own, admitted like a batch); with final
 *   != 0 the hash of every byte appended so far is written to host_out (one
 *   uint32 or uint64) and the string may still be extended afterwards. The
 *   pieces of one string are applied in submission order, whichever slots
 *   run them. PMP_EINVAL for an unknown stream; a piece that would make the
 *   string longer than 8 tree levels cover fails its ticket with
 *   PMP_ETOOLONG.
 * pmp_server_stream_close: waits until the string's pieces are issued,
 *   synchronizes the device and frees the string's state.
 * pmp_server_wait: waits up to timeout_s (0 <= timeout_s; larger than 1e9 is
 *   taken as 1e9; a negative or NaN timeout is PMP_EINVAL) for a ticket;
 *   *done tells whether it finished; returns the request's status: PMP_OK,
 *   an error of issuing it (PMP_ECUDA, PMP_ETOOLONG, ...) or a device-side
 *   error of its own batch call (PMP_ESCRATCH, PMP_ETIMEOUT).
 * pmp_server_ticket_times: steady-clock nanoseconds of submission, admission
 *   and completion (results visible on the host) of a ticket.
 * pmp_server_release: forget a finished ticket.
 * pmp_server_destroy: stops the scheduler (requests still queued are
 *   dropped; wait for them first), frees the arena, the streams and the
 *   strings still open.
 * ------------------------------------------------------------------------- */
typedef struct pmp_server pmp_server;
int pmp_server_create(const pmp_key *key32, const pmp_key *key64, size_t budget_bytes, int slots,
                      pmp_server **out);
int pmp_server_submit(pmp_server *s, int width, const uint8_t *host_base,
                      const int64_t *host_offsets, int64_t n, void *host_out, uint64_t *ticket);
int pmp_server_stream_open(pmp_server *s, int width, uint64_t *stream_id);
int pmp_server_submit_piece(pmp_server *s, uint64_t stream_id, const void *host_piece, uint64_t len,
                            int final, void *host_out, uint64_t *ticket);
int pmp_server_stream_close(pmp_server *s, uint64_t stream_id);
int pmp_server_wait(pmp_server *s, uint64_t ticket, double timeout_s, int *done);
int pmp_server_ticket_times(pmp_server *s, uint64_t ticket, uint64_t *submit_ns,
                            uint64_t *start_ns, uint64_t *done_ns);
int pmp_server_release(pmp_server *s, uint64_t ticket);
void pmp_server_destroy(pmp_server *s);

/* ---------------------------------------------------------------------------
 * Streaming: one string hashed from pieces that arrive one after another.
 * Sec. 4 notes that the tree of Algorithm 1 can be evaluated while the string
 * is read once, keeping one incomplete chunk per level; here that running
 * state lives in device memory owned by the stream object, and each update
 * hashes its complete level-1 chunks and folds them into the levels above in
 * parallel. The result equals pmp_hash32/64 of the concatenated pieces.
 *
 * pmp_stream_create: state for one string with `key` (its width decides the
 *   output: uint32 for a 32-bit key, uint64 for 64). Allocates about 1 MiB of
 *   device memory on the current device; the key must outlive the stream.
 *   PMP_ENOMEM if the allocation fails.
 * pmp_stream_update: appends len bytes at d_piece (device memory, any
 *   alignment and length; the aligned 8-byte words that hold its first and
 *   last bytes are read whole, the bytes outside the piece ignored). Work is
 *   queued on `stream` (NULL = default stream); the piece must stay valid
 *   and unchanged until it has run. PMP_ETOOLONG if the string would exceed
 *   what an 8-level tree covers (as for pmp_hash32/64); nothing is appended
 *   then. An update of whole level-2 chunks (a piece that starts a level-2
 *   chunk: m^2 words) is one tree-kernel launch that lets programmatic
 *   dependents start once all its tile claims are made, and that is itself
 *   a programmatic dependent of the kernel before it, so consecutive such
 *   updates overlap. Stream order holds for every other operation. A kernel
 *   the caller launches right after an update with programmatic stream
 *   serialization may start before the update has finished: it must wait
 *   for its prerequisite grid (cudaGridDependencySynchronize) before it
 *   touches the piece, as that attribute requires.
 * pmp_stream_final: writes the hash of the bytes appended so far to d_out
 *   (one uint32 or uint64) and, if d_raw is not NULL, the tree value before
 *   the output step to d_raw[0..1] (low 64 bits, high bit). Queued on
 *   `stream`; the state is unchanged, so updates may continue the string.
 * pmp_stream_reset: starts a new (empty) string, queued on `stream`.
 * pmp_stream_length: bytes appended so far (host-side count).
 * pmp_stream_destroy: synchronizes the device and frees the state.
 * Calls on one stream object must come from one host thread at a time and be
 * issued on one CUDA stream (or otherwise ordered).
 * ------------------------------------------------------------------------- */
typedef struct pmp_stream pmp_stream;
int pmp_stream_create(const pmp_key *key, pmp_stream **out);
int pmp_stream_update(pmp_stream *s, const void *d_piece, uint64_t len, void *stream);
int pmp_stream_final(pmp_stream *s, void *d_out, uint64_t *d_raw, void *stream);
int pmp_stream_reset(pmp_stream *s, void *stream);
uint64_t pmp_stream_length(const pmp_stream *s);
void pmp_stream_destroy(pmp_stream *s);

/* ---------------------------------------------------------------------------
 * Tuning knobs (process-wide, not part of the paper): set by the autotuner
 * (paper_1609_09840_gb300/autotune.py), which times the choices on the
 * current GPU and caches the winners. Results never depend on them.
 *   PMP_KNOB_TREE_STAGES_32/64: TMA staging depth of the single-buffer tree
 *     kernel (2, 3, 4 or 6 stages of 16 KiB; default 4).
 *   PMP_KNOB_BATCH_SCHED: schedule of the batch's one-chunk strings:
 *     PMP_BATCH_SORTED (default): ranges of strings staged in shared
 *     memory by bulk copies and sorted by length, a warp hashing 32 strings
 *     of nearly equal length, one lane each; PMP_BATCH_TILES: tiles of 64
 *     consecutive strings read from global memory, one lane per string for
 *     the first units, the rest in pieces dealt out to the warp.
 *   PMP_KNOB_BATCH_RANGE: strings per range of the sorted schedule: 512
 *     (blocks of 4 warps, 28 KiB staged per fill) or 1024 (blocks of 8
 *     warps, 56 KiB per fill; default).
 *   PMP_KNOB_CHUNK_STAGES_32/64: staging depth of the chunk kernel that
 *     hashes a batch's strings of 32 or more level-1 chunks, per width: 2 (4
 *     blocks per SM; default) or 3 (3 blocks per SM).
 *   PMP_KNOB_STREAM_SEGMENT: level-1 chunks per segment of a streaming
 *     update (2^17, 2^18 or 2^19; default 2^19): a piece is hashed in
 *     segments of at most this many chunks, a few launches each.
 *   PMP_KNOB_BATCH_P1: 8-byte units of every string that the tile schedule's
 *     first pass takes with one lane per string (6 or 8; longer strings
 *     continue in 4-unit pieces dealt out to the warp; default 6).
 * pmp_tune_set returns PMP_EINVAL for an unknown knob or value.
 * ------------------------------------------------------------------------- */
enum {
    PMP_KNOB_TREE_STAGES_32 = 0,
    PMP_KNOB_TREE_STAGES_64 = 1,
    PMP_KNOB_BATCH_P1 = 2,
    PMP_KNOB_BATCH_SCHED = 3,
    PMP_KNOB_BATCH_RANGE = 4,
    PMP_KNOB_CHUNK_STAGES_32 = 5,
    PMP_KNOB_STREAM_SEGMENT = 6,
    PMP_KNOB_CHUNK_STAGES_64 = 7
};
enum { PMP_BATCH_SORTED = 0, PMP_BATCH_TILES = 1 };
int pmp_tune_set(int knob, int value);
int pmp_tune_get(int knob, int *value);

/* Read and clear the device status word of the current device (synchronizes
 * the device). *out receives PMP_OK or the first device-side error code. */
int pmp_device_status(int *out);

/* Static description of a status code. */
const char *pmp_strerror(int status);

#ifdef __cplusplus
}
#endif
#endif /* PMPLUS_H */
