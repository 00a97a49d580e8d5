/*
 * rfr.h — C ABI of the RFR (Real-Factors-Recombination) factorisation library
 * for NVIDIA B300 (sm_103a).
 *
 * The library factors a monic, square-free polynomial p in Z[x] into its
 * monic irreducible factors by the method of "Integer polynomial
 * factorization by recombination of real factors" (arXiv 2410.15880):
 *   1. all complex roots of p (Section 2, "black box"; here a batched FP64
 *      Aberth iteration with a double-double Newton polish and an inclusion
 *      radius per root),
 *   2. the real factorisation of Eq. 1 and the fractional parts rho of the
 *      first traces (Section 2), scaled to 64-bit fixed point (Eq. 18),
 *   3. the meet-in-the-middle subset-sum search of Section 3.3 (Horowitz-
 *      Sahni): all half-subset sums of each half, sorted, and matched
 *      against the integrality window of Eq. 9 / Eq. 19,
 *   4. the candidate test of Algorithm FACTOR (q in Z[x]) by rounding and
 *      exact integer division, and the irreducible factors as atoms of the
 *      verified divisors.
 * Every step runs in CUDA kernels on one GPU; the host code only validates,
 * plans memory, launches and assembles results.
 *
 * Conventions shared by every call
 *  - Polynomials are arrays of int64 coefficients in ASCENDING powers:
 *    coeffs[0] = a_0 ... coeffs[degree] = a_degree.  The input must be monic
 *    (coeffs[degree] == 1), 1 <= degree <= RFR_MAX_DEGREE and |a_i| < 2^53.
 *  - Status codes: RFR_OK (0) on success, RFR_PENDING (> 0) for a request
 *    still in flight, negative RFR_E_* values on error.  No call aborts the
 *    process; every call is thread-safe with respect to one context.
 *  - Input buffers are read (and copied where the call returns before the
 *    work ends) before the call returns; the caller keeps ownership.
 *  - Output factor lists are allocated by the library and released by the
 *    caller with rfr_factors_free().
 */
#ifndef RFR_H_
#define RFR_H_

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define RFR_MAX_DEGREE 128

/* ---- status codes ------------------------------------------------------ */
#define RFR_OK                 0
#define RFR_PENDING            1   /* rfr_poll: request not finished yet      */
#define RFR_E_INVALID         -1   /* null pointer / bad argument / unknown ticket */
#define RFR_E_NOT_MONIC       -2   /* coeffs[degree] != 1                     */
#define RFR_E_RANGE           -3   /* degree outside [1,128] or |a_i| >= 2^53 */
#define RFR_E_NOT_SQUAREFREE  -4   /* p and p' share a factor (Section 2 assumes square-free) */
#define RFR_E_NO_CONVERGENCE  -5   /* root iteration did not converge         */
#define RFR_E_ROOTS           -6   /* inclusion discs overlap or real/complex classification undecidable */
#define RFR_E_WINDOW          -7   /* integrality window too wide for the search */
#define RFR_E_CAND_OVERFLOW   -8   /* more candidate patterns than the configured cap */
#define RFR_E_OVERFLOW        -9   /* a verified candidate needs more than int128 / |c| < 2^62 */
#define RFR_E_OOM            -10   /* device or host allocation failed        */
#define RFR_E_BUDGET         -11   /* the request's tables exceed the memory budget */
#define RFR_E_TIMEOUT        -12   /* rfr_wait timed out (request still queued/running) */
#define RFR_E_CUDA           -13   /* a CUDA runtime call failed              */
#define RFR_E_CANCELLED      -14   /* request cancelled with rfr_cancel       */
#define RFR_E_INTERNAL       -15   /* an internal consistency check failed    */

/* ---- root finder precision (rfr_config.root_mode) ----------------------- */
#define RFR_ROOTS_FP64       0     /* Aberth in FP64, then double-double polish */
#define RFR_ROOTS_FP32_BULK  1     /* Aberth bulk in FP32, then FP64, then double-double polish */

typedef struct rfr_ctx rfr_ctx;   /* opaque: owns streams, device memory, worker threads */

/* Library configuration.  Fill with rfr_config_default() and override. */
typedef struct {
    int      device;            /* CUDA device ordinal                                   */
    size_t   mem_budget_bytes;  /* device bytes the context may hold for tables; 0 = 85% of free memory at create */
    int      max_inflight;      /* serving: batches that may run concurrently (streams), >= 1 */
    int      max_batch;         /* serving: requests admitted into one batch                */
    int      root_mode;         /* RFR_ROOTS_FP64 or RFR_ROOTS_FP32_BULK                    */
    int      timing;            /* 1: record CUDA events per stage into rfr_diag.stage_us   */
    uint64_t max_candidates;    /* per polynomial cap on candidate patterns (after the Tr_1/Tr_2 windows) */
    double   eps_override;      /* > 0: integrality window eps (fraction of 1) replacing the derived one */
    int      use_graphs;        /* 1: replay the batch prologue (copy in, validate, roots, weights,
                                   plans out) as a captured CUDA graph per batch size (host inputs),
                                   and the match of a sub-batch of fused-match problems (job upload,
                                   sorted lists, k_mitm, exact re-check, compaction) as a captured
                                   graph per launch shape, captured when a shape occurs the second
                                   time in a pipeline; both for caller batches only (blocking,
                                   device and asynchronous calls), not the batches formed from the
                                   request queue, whose sizes and compositions rarely recur */
    int      autotune;          /* 1: time candidate layouts on the first problem of each (n_a, n_b)
                                   class and keep the best: for the fused match the key-unit size
                                   (2^12 .. 2^14 half-a keys per unit) and the bin limit, for the
                                   table match the low-list bits, bucket digit and CTAs per SM */
    const char* tune_cache_path;/* NULL, or a text file that stores tuned layouts across runs (read at
                                   create, appended when a class is tuned); the string is copied */
    int      match_path;        /* RFR_MATCH_AUTO: halves of n_b <= 13 in one shared-memory kernel,
                                   14 <= n_a <= n_b <= 32 by the fused match, the rest by the table
                                   match; RFR_MATCH_TABLES: every problem with n_b > 13 by the
                                   table match with the count-pass layout; RFR_MATCH_SPLAT: every
                                   problem with 13 < n_b <= 30 by the splat match (Section 4,
                                   Algorithm E), falling back to the table match when an insertion
                                   overflows; RFR_MATCH_PRUNE: every problem with n_b > 13 and
                                   n_a + n_b <= 40 by Algorithm B's pruned search (Section 3.2)
                                   (same results on every path)                                    */
    int      reserved0;
} rfr_config;

/* rfr_config.match_path */
#define RFR_MATCH_AUTO   0
#define RFR_MATCH_TABLES 1
#define RFR_MATCH_SPLAT  2
#define RFR_MATCH_PRUNE  3

/* Per-polynomial diagnostics returned with each result.  The stage times,
 * copy bytes and launch count describe the whole batch the polynomial was
 * factored in (batch_size polynomials); stage times are CUDA-event times on
 * the batch's stream, filled when rfr_config.timing is set. */
typedef struct {
    int      n, r, c;           /* n = r + c elements of Eq. 1: r real roots, c conjugate pairs */
    int      n_a, n_b;          /* half sizes of the meet-in-the-middle split (one element fixed out) */
    uint64_t window;            /* Tr_1 window W in units of 2^-64                          */
    uint64_t half_sums;         /* 2^n_a + 2^n_b table entries enumerated                    */
    uint64_t cand_coarse;       /* pairs within the coarse (prefix) window                   */
    uint64_t cand_pre;          /* pairs within the exact Tr_1 window W                      */
    uint64_t cand_post;         /* ... that also pass the Tr_2 window                        */
    uint64_t verified;          /* candidates proven to divide p                             */
    double   max_rel_residual;  /* max_i |p(z_i)| / sum_k |a_k||z_i|^k after the polish       */
    double   max_root_err;      /* largest inclusion radius                                  */
    double   stage_us[8];       /* validate+roots, weights, sorted lists (+ count pass and scans of
                                   the table match), table scatter, match (table join and/or
                                   the fused match), verify+atoms, device total, host total (us) */
    uint64_t h2d_bytes;         /* bytes the batch copied host -> device                     */
    uint64_t d2h_bytes;         /* bytes the batch copied device -> host                     */
    uint32_t launches;          /* CUDA kernels the batch launched                           */
    uint32_t batch_size;        /* polynomials in the batch                                  */
    uint32_t graphs;            /* captured CUDA graphs the batch replayed (prologue, match)  */
    uint32_t reserved;
} rfr_diag;

/* A factorisation: n_factors monic irreducible factors in canonical order
 * (degree ascending, then (a_0, ..., a_{e-1}) lexicographic as signed int64).
 * degrees[i] is the degree of factor i; coeffs holds the factors one after
 * the other, each as degree+1 ascending coefficients (monic).  The product of
 * the factors equals the input exactly. */
typedef struct {
    int      n_factors;
    int*     degrees;
    int64_t* coeffs;
    rfr_diag diag;
} rfr_factors;

/* A factorisation of any nonzero p in Z[x] (rfr_factor_general):
 * p = content * prod_i f_i^multiplicities[i], each f_i primitive,
 * irreducible over Z and with a positive leading coefficient (content
 * carries the sign), in canonical order (degree ascending, then the
 * coefficients a_0 .. a_e lexicographic as signed int64, then the
 * multiplicity).  coeffs holds the f_i one after the other, degrees[i] + 1
 * ascending coefficients each.  rfr_squarefree fills the same structure
 * with the square-free parts instead (each f_i square-free, not necessarily
 * irreducible, pairwise coprime, distinct multiplicities apart from the
 * factor x). */
typedef struct {
    int64_t  content;
    int      n_factors;
    int*     degrees;
    int*     multiplicities;
    int64_t* coeffs;
} rfr_factorization;

/* Device allocator hook (e.g. PyTorch's caching allocator).  alloc returns a
 * device pointer of at least `bytes` bytes usable on `stream` (a
 * cudaStream_t), or NULL; free releases it. */
typedef void* (*rfr_alloc_fn)(size_t bytes, void* user, void* stream);
typedef void  (*rfr_free_fn)(void* ptr, size_t bytes, void* user, void* stream);

/* Fill *cfg with defaults: device 0, budget 0 (auto), max_inflight 2,
 * max_batch 64, FP32-bulk roots, timing off, 1<<16 candidates, no override,
 * graphs on, autotune off, no tune cache file.
 * Returns RFR_E_INVALID if cfg is NULL. */
int rfr_config_default(rfr_config* cfg);

/* Create a context on cfg->device (cfg may be NULL for defaults).  Errors:
 * RFR_E_INVALID (bad config), RFR_E_CUDA (device unusable). */
int rfr_create(const rfr_config* cfg, rfr_ctx** out);

/* Stop the serving workers (pending requests end RFR_E_CANCELLED), free all
 * device memory and destroy the context.  NULL is accepted. */
int rfr_destroy(rfr_ctx* ctx);

/* Route the context's device allocations through alloc/free (both non-NULL),
 * or back to the built-in stream-ordered pool (both NULL).  Must be called
 * while no request is in flight; returns RFR_E_INVALID otherwise. */
int rfr_set_allocator(rfr_ctx* ctx, rfr_alloc_fn alloc, rfr_free_fn free_fn, void* user);

/* Factor one polynomial (blocking).  On RFR_OK *out holds the factors; on
 * error *out is zeroed except out->diag.  Algorithm FACTOR, Section 2. */
int rfr_factor(rfr_ctx* ctx, const int64_t* coeffs, int degree, rfr_factors* out);

/* Factor any nonzero p in Z[x] of degree <= 128 (blocking), by the
 * reductions Section 2 names: content and sign, the power of x, the monic
 * transform q(y) = lc^(d-1) p(y / lc), Yun's square-free decomposition of q
 * (modulo 61-bit primes, lifted and checked exactly), the GPU factorisation
 * of every square-free part as one batch, and the back transform (primitive
 * part of g(lc x)).  content * prod f^m == p is checked exactly.
 * Errors: RFR_E_INVALID (NULL, zero polynomial, degree outside 0..128),
 * RFR_E_RANGE (a transformed part has a coefficient of 2^53 or more),
 * RFR_E_OVERFLOW (a lift or a back transform leaves 128-bit or int64
 * range), and the errors of rfr_factor_batch.  Free *out with
 * rfr_factorization_free. */
int rfr_factor_general(rfr_ctx* ctx, const int64_t* coeffs, int degree, rfr_factorization* out);

/* Square-free decomposition only (steps above up to Yun, mapped back to p),
 * on the host: needs no context and no GPU. */
int rfr_squarefree(const int64_t* coeffs, int degree, rfr_factorization* out);

/* Free what rfr_factor_general / rfr_squarefree allocated; zeroes *f.
 * NULL and zeroed structures are accepted. */
void rfr_factorization_free(rfr_factorization* f);

/* Factor `count` polynomials as one batch (blocking): the stages run once
 * over the whole batch.  coeffs[i] points at degrees[i]+1 coefficients.
 * outs[i] / statuses[i] receive each result.  The return value is RFR_OK if
 * the batch ran (individual statuses may still be errors), else the error
 * that stopped the whole batch. */
int rfr_factor_batch(rfr_ctx* ctx, int count, const int64_t* const* coeffs,
                     const int* degrees, rfr_factors* outs, int* statuses);

/* Key-range sharding of one batch over nshards processes (one per GPU),
 * each calling this with its own shard index (0 .. nshards-1) on the same
 * inputs.  The fused match of every problem searches only this shard's
 * contiguous share of the key units (the slabs of half a's key space); the
 * other matches (small halves, table match) run on shard 0, and a problem
 * that a shard redoes with the table match is searched whole there.  After
 * verifying its own candidates, every shard calls gather once (even with
 * nothing to send):
 *   mine/n_mine: this shard's verified divisor sets as n_mine triples
 *   (item index, pattern bits 0-63, pattern bits 64-127);
 *   *all/*n_all: the caller returns every shard's triples (malloc'ed; the
 *   library frees them), e.g. an all-gather over a process group.
 * gather returns 0, or non-zero to fail the batch (RFR_E_INVALID).  Every
 * shard then builds the atoms from the union, so all shards return the same
 * factorisation.  A shard whose batch fails before the gather does not call
 * it: give the exchange a timeout.  nshards == 1 is rfr_factor_batch. */
typedef int (*rfr_gather_fn)(const uint64_t* mine, size_t n_mine, uint64_t** all, size_t* n_all, void* user);
int rfr_factor_batch_sharded(rfr_ctx* ctx, int count, const int64_t* const* coeffs, const int* degrees,
                             int shard, int nshards, rfr_gather_fn gather, void* user,
                             rfr_factors* outs, int* statuses);

/* As rfr_factor_batch, for inputs already in device memory:
 * d_coeffs is int64 [count][RFR_MAX_DEGREE+1] (ascending, row i holds
 * polynomial i, entries above its degree ignored) and d_degrees int32
 * [count], both device pointers valid until the call returns.  Input
 * checks run on the device.  Results are returned in host memory as for
 * rfr_factor_batch. */
int rfr_factor_batch_device(rfr_ctx* ctx, int count, const int64_t* d_coeffs,
                            const int32_t* d_degrees, rfr_factors* outs, int* statuses);

/* rfr_factor_batch without blocking: the batch is queued whole for one of
 * the serving workers (ahead of single requests) and runs on that worker's
 * pipeline and stream, so the caller can prepare the next batch, or read the
 * last one's results, while this one runs; batches queued back to back run
 * on different workers and overlap on the device.  The rows are copied
 * before the call returns.  outs[count] and statuses[count] (statuses may be
 * NULL) belong to the caller and must stay valid until rfr_batch_wait has
 * returned for *ticket; they are zeroed / set to RFR_PENDING here.
 * Returns RFR_OK with *ticket set, or RFR_E_INVALID (bad arguments, a context
 * without workers, or one being destroyed). */
int rfr_factor_batch_async(rfr_ctx* ctx, int count, const int64_t* const* coeffs, const int* degrees,
                           rfr_factors* outs, int* statuses, uint64_t* ticket);

/* Wait for a batch queued by rfr_factor_batch_async (timeout_ms < 0: no
 * limit).  Returns what rfr_factor_batch would have returned, with outs /
 * statuses filled the same way, and releases the ticket; RFR_E_TIMEOUT
 * leaves the batch in place (wait again); RFR_E_INVALID for an unknown or
 * released ticket.  rfr_destroy drops batches still queued (their statuses
 * become RFR_E_CANCELLED) and waits for running ones: wait for every batch
 * before destroying its context. */
int rfr_batch_wait(rfr_ctx* ctx, uint64_t ticket, int timeout_ms);

/* Serving API (continuous batching).  rfr_submit copies the input and
 * queues it; workers admit queued requests into batches as slots and device
 * memory free up, and batches in flight overlap on the device.
 * *ticket identifies the request.  Input errors (monic, range) are reported
 * at submit time. */
int rfr_submit(rfr_ctx* ctx, const int64_t* coeffs, int degree, uint64_t* ticket);

/* Non-blocking: RFR_PENDING while queued or running; otherwise the
 * request's final status, with *out filled on RFR_OK.  A finished ticket
 * is released by the first rfr_poll/rfr_wait that returns its result. */
int rfr_poll(rfr_ctx* ctx, uint64_t ticket, rfr_factors* out);

/* rfr_poll for n tickets under one lock: statuses[i] is RFR_PENDING or the
 * request's final status (outs[i] filled on RFR_OK, ticket released), or
 * RFR_E_INVALID for an unknown ticket.  Returns RFR_OK, or RFR_E_INVALID on
 * bad arguments.  For clients that track many requests at once. */
int rfr_poll_batch(rfr_ctx* ctx, int n, const uint64_t* tickets, rfr_factors* outs, int* statuses);

/* Block until the request finishes or timeout_ms elapses (< 0: no limit);
 * RFR_E_TIMEOUT leaves the request in place. */
int rfr_wait(rfr_ctx* ctx, uint64_t ticket, int timeout_ms, rfr_factors* out);

/* Cancel a queued request (it then finishes with RFR_E_CANCELLED).  A request
 * already running completes normally.  RFR_E_INVALID for unknown tickets. */
int rfr_cancel(rfr_ctx* ctx, uint64_t ticket);

/* Release the arrays of a result; safe on a zeroed or already freed struct. */
void rfr_factors_free(rfr_factors* f);

/* rfr_factors_free on each of f[0 .. count) (the results of one batch call). */
void rfr_factors_free_n(rfr_factors* f, int count);

/* Copy the factors of f[0 .. count) (the results of one batch call) into flat
 * caller arrays: n_factors[i] = f[i].n_factors; the degrees of all factors,
 * result by result, into degrees[]; their coefficients, one factor after the
 * other, into coeffs[].  Nothing is freed.  Returns the number of
 * coefficients written, RFR_E_RANGE if coeffs_cap or degrees_cap is too
 * small (the arrays are then partly written), RFR_E_INVALID on bad
 * arguments.  The factors of a degree-d polynomial hold at most 2 (d + 1)
 * coefficients. */
int64_t rfr_factors_flatten(rfr_factors* f, int count, int64_t* coeffs, size_t coeffs_cap,
                            int32_t* degrees, size_t degrees_cap, int32_t* n_factors);

/* Static English description of a status code. */
const char* rfr_strerror(int status);

/* Library version string. */
const char* rfr_version(void);

#ifdef __cplusplus
}
#endif
#endif /* RFR_H_ */
