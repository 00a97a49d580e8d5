/*
 * rfr_stages.h — stage-level C ABI of the RFR library (device pointers).
 *
 * These entry points run one stage of the hot path on buffers that already
 * live in device memory, on the caller's CUDA stream (passed as void*, a
 * cudaStream_t; NULL = the legacy default stream).  They exist so that each
 * stage can be checked on its own against the CPU oracle and timed on its
 * own; rfr_factor / rfr_factor_batch in rfr.h chain the same kernels.
 * All pointers are device pointers unless named h_*; the caller owns every
 * buffer.  Calls are asynchronous: they return after the launches are
 * queued (RFR_OK) or with RFR_E_INVALID for bad sizes and RFR_E_CUDA if a
 * launch failed.  Errors found by the kernels are written to the stated
 * device status words.
 */
#ifndef RFR_STAGES_H_
#define RFR_STAGES_H_

#include <stddef.h>
#include <stdint.h>
#include "rfr.h"

#ifdef __cplusplus
extern "C" {
#endif

/* Coefficient layout for the stages: int64 [batch][RFR_LDC], ascending
 * powers, entries above each problem's degree ignored. */
#define RFR_LDC (RFR_MAX_DEGREE + 1)

/* Status value of the validate and roots stages: square-free not proven
 * modulo primes; the roots stage decides (disjoint inclusion discs prove
 * distinct roots) and reports RFR_E_NOT_SQUAREFREE if it cannot separate
 * them.  Never returned by the rfr.h calls. */
#define RFR_SF_SUSPECT 2

/* Per-polynomial plan written by the weights stage (one per problem).
 * Elements are the factors of Eq. 1 in canonical order: real roots
 * ascending, then conjugate pairs by (Re z, Im z) of the member with
 * Im z > 0.  The last element (index n-1) is fixed out of the search
 * (complement symmetry, Section 3.1); elements 0..n_a-1 form half a and
 * n_a..n_a+n_b-1 half b. */
typedef struct {
    int32_t  status;        /* RFR_OK or the first error of roots/weights     */
    int32_t  degree;
    int32_t  n, r, c;       /* elements, real roots, conjugate pairs          */
    int32_t  n_a, n_b;      /* n_a = floor((n-1)/2), n_b = n-1-n_a            */
    int32_t  pad0;
    uint64_t window;        /* Tr_1 window W (units of 2^-64)                 */
    uint64_t window2;       /* Tr_2 window W2 (units of 2^-64; >= 2^63 = off) */
    double   max_radius;    /* largest root inclusion radius                  */
    double   max_rel_residual;
    double   sum_err1;      /* bound on |error| of any Tr_1 subset sum        */
    double   sum_err2;      /* same for Tr_2                                  */
    uint64_t w[RFR_MAX_DEGREE];    /* rho_k scaled: round(frac(Tr_1 part) * 2^64) mod 2^64 (Eq. 18) */
    uint64_t w2[RFR_MAX_DEGREE];   /* Tr_2 part scaled the same way           */
    uint8_t  kind[RFR_MAX_DEGREE]; /* 1 = real linear factor, 2 = real quadratic factor */
    uint8_t  root0[RFR_MAX_DEGREE];/* root index (into the roots array) of element k    */
    uint8_t  root1[RFR_MAX_DEGREE];/* conjugate partner's root index (pairs only)       */
} rfr_plan;

/* K-v validate.  status[i] = RFR_OK, RFR_SF_SUSPECT, RFR_E_RANGE (degree
 * outside [1,128] or |a_k| >= 2^53) or RFR_E_NOT_MONIC for the polynomial
 * coeffs[i*RFR_LDC ..] of degree degrees[i].  Square-free is proven when
 * gcd(p, p') is constant modulo 2^31-1 or 2^61-1 (Section 2 assumes
 * square-free input). */
int rfr_stage_validate(const int64_t* coeffs, const int32_t* degrees, int batch,
                       int32_t* status, void* stream);

/* K-a roots.  For problem i (degree degrees[i]) writes its roots to
 * roots[i*RFR_MAX_DEGREE*4 + 4*j + {0,1,2,3}] = (Re hi, Re lo, Im hi, Im lo)
 * as double-double values, the inclusion radius of root j to
 * radius[i*RFR_MAX_DEGREE + j] (a disc of that radius around the root
 * contains exactly one root of p when the discs are disjoint), and RFR_OK,
 * RFR_E_NO_CONVERGENCE or RFR_E_RANGE to status[i].  status is in/out: on
 * entry a negative value skips problem i (kept), RFR_SF_SUSPECT is carried
 * through (and turns non-convergence into RFR_E_NOT_SQUAREFREE), anything
 * else must be RFR_OK.
 * root_mode: RFR_ROOTS_FP64 or RFR_ROOTS_FP32_BULK.  Section 2, Eq. 1. */
int rfr_stage_roots(const int64_t* coeffs, const int32_t* degrees, int batch,
                    int root_mode, double* roots, double* radius,
                    int32_t* status, void* stream);

/* K-b weights.  From the roots and radii of K-a, classify real roots and
 * conjugate pairs (Eq. 1), order the elements, and write plans[i]: the
 * fixed-point Tr_1 weights w (Eq. 18, rounded), Tr_2 weights w2, the
 * windows W and W2 derived from the radii, and the half split.
 * eps_override > 0 replaces W by ceil(eps_override * 2^64).  Section 2,
 * Section 3.3. */
int rfr_stage_weights(const int64_t* coeffs, const int32_t* degrees, int batch,
                      const double* roots, const double* radius,
                      const int32_t* root_status, double eps_override,
                      rfr_plan* plans, void* stream);

/* K-c, plain form: keys[s] = (sum of w[i] over the set bits i of s) mod 2^64
 * for s = 0 .. 2^h - 1, written in pattern order with 128-bit stores
 * (EXPAND before its sort, Section 3.3).  1 <= h <= 32 (h = 0 writes the
 * single entry 0).  keys must hold 2^h entries, 16-byte aligned. */
int rfr_stage_enumerate(const uint64_t* w, int h, uint64_t* keys, void* stream);

/* Match workspace: bytes of device scratch rfr_stage_match needs for halves
 * of n_a and n_b elements. */
size_t rfr_stage_match_workspace(int n_a, int n_b);

/* Bytes of device scratch rfr_stage_match_fused needs for halves of n_a and
 * n_b elements (2 <= n_a <= n_b <= 32): its sorted lists, their masks and
 * directories, and room for 2^20 fingerprint hits; 0 if the fused match does
 * not take these halves.  Section 3.3. */
size_t rfr_stage_match_fused_workspace(int n_a, int n_b);

/* K-d for the fused match: one half's sorted list of low-subset sums.
 * For every subset s of the weights w[0..l), list[] receives the exact sum
 * S(s) = sum over i in s of w_i modulo 2^64 (of -w_i when negate != 0) and
 * masks[] the subset s at the same position; list is ascending as uint64
 * (ties in any order).  0 <= l <= 25; workspace:
 * rfr_stage_lowlist_workspace(l) bytes, 256-byte aligned; list: 2^l uint64,
 * masks: 2^l uint32, both caller-owned device memory.  Built by merging: the
 * list of i elements and its copy shifted by w_i (rotated where the shifted
 * sums wrap past 2^64), with bit i added to the copy's masks (EXPAND's sort,
 * Section 3.3).  RFR_E_INVALID for null pointers, l out of range, an
 * unaligned or short workspace. */
size_t rfr_stage_lowlist_workspace(int l);
int rfr_stage_lowlist(const uint64_t* w, int l, int negate, uint64_t* list, uint32_t* masks,
                      void* workspace, size_t workspace_bytes, void* stream);

/* K-d + K-e as the paper designs them for the GPU (Section 4, Algorithm E):
 * SPLAT of half b (Algorithm D, c = 2, with the atomic-exchange INSERT of
 * Section 4) and a band QUERY from every pattern of half a.
 *
 * gamma: caller-owned device buffer of rfr_stage_splat_cells(n_b) uint64
 * cells, 256-byte aligned (0 if n_b is outside 0..30).  After either call its
 * first 2^(n_b+1) + 4096 cells hold the splat array: cell i is ~0 (empty) or
 * e(s) = ((S_b(s) >> 1) & ~(2^n_b - 1)) | s for a pattern s of half b with
 * S_b(s) = sum_{j in s} w_b[j] mod 2^64.  Each e(s) sits at or after its home
 * cell e(s) >> (62 - n_b), every cell in between is full, and the full cells
 * are increasing in index order (the step past a full cell is linear, into
 * 4096 overflow cells, instead of the paper's circular step).  The last 256
 * bytes hold the launch descriptor.
 * counters: 8 device words, zeroed by the call:
 *   [0] cells within a scanned range   [1] pairs within W (Eq. 9, circular)
 *   [2] candidates (also within W2 for the w2 weights, not the empty pair)
 *   [3] 1 when the empty pair was met  [4] 1 when an insertion ran past the
 *   overflow cells or its step limit (the array then misses values)
 *   [5] cells INSERT looked at (Theorem 3.4.2's C = [5] / 2^n_b)
 *   [6] atomic exchanges                [7] cells QUERY read
 * Candidates are s_a | s_b << n_a, at most cap of them written (any order).
 * QUERY reports every pair in the window: the printed QUERY stops at its
 * first hit and starts at the target's home cell, which misses pairs. */
size_t rfr_stage_splat_cells(int n_b);
int rfr_stage_splat(const uint64_t* w_b, int n_b, uint64_t* gamma, size_t gamma_cells,
                    unsigned long long* counters, void* stream);
int rfr_stage_splat_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                          const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                          uint64_t window, uint64_t window2, uint64_t* gamma, size_t gamma_cells,
                          uint64_t* cand, uint64_t cap, unsigned long long* counters, void* stream);

/* Algorithm B (Section 3.2, RECOMBINE_B): every pattern s of the m searched
 * elements w[0..m) (the fixed element left out) with
 * dist(sum_{i in s} w_i mod 2^64) <= window (Eq. 9, circular), found by the
 * pruned search: the elements are sorted ascending, and after a pattern with
 * value x the search jumps over the next 2^j - 1 patterns when their values,
 * all in [x + w_min, x + (sum of the j smallest)], miss both acceptance
 * bands.  0 <= m <= 44 (the work is about 2^m / (2^l / l), l =
 * floor(sqrt(2m)), Theorem 3.2.1).  Candidates are the accepted non-empty
 * patterns whose w2 sum is within window2, as bit masks over w's order, at
 * most cap written (any order).  counters: 8 device words, zeroed by the call:
 * [0] patterns visited, [1] patterns within W (the empty one included),
 * [2] candidates, [3] 1 when the empty pattern was met.
 * workspace: 256 device bytes, 256-byte aligned (the launch descriptor). */
int rfr_stage_prune(const uint64_t* w, const uint64_t* w2, int m, uint64_t window, uint64_t window2,
                    uint64_t* cand, uint64_t cap, unsigned long long* counters,
                    void* workspace, size_t workspace_bytes, void* stream);

/* K-c + K-d + K-e for one problem given its weights: enumerate both halves
 * (keys of half b negated), radix-partition them by key (first digit fused
 * into the enumeration, second digit in shared memory inside the match),
 * and write every pattern s = s_a | (s_b << n_a), s != 0, with
 *   dist((sum_a w_a + sum_b w_b) mod 2^64) <= W   and
 *   dist((sum_a w2_a + sum_b w2_b) mod 2^64) <= W2,
 * dist(y) = min(y, 2^64 - y) (Eq. 9 / Eq. 19 made circular), to
 * cand[0 .. min(count, cap)).  counters (device, uint64 [6]) receive
 * {coarse pairs, pairs within W, pairs also within W2 (= count), trivial
 * pattern seen (1/0), layout overflow (1/0), fingerprint hits of the fused
 * match (0 for the other matches)}.  w_a/w2_a hold n_a weights, w_b/w2_b n_b; 0 <= n_a,
 * n_b <= 32.  workspace: rfr_stage_match_workspace(n_a, n_b) bytes,
 * 256-byte aligned.  Section 3.3 (RECOMBINE_C's result set).
 * Tables of half b with n_b <= 13 are matched in one shared-memory kernel.
 * Larger ones use per-bucket regions with 25 % slack over the mean count
 * (no count pass); if keys cluster so that a region or a halo list fills up,
 * counters[4] is set to 1 and the candidates are incomplete: the caller then
 * runs rfr_stage_match_exact, which sizes every bucket with a count pass. */
int rfr_stage_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                    const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                    uint64_t window, uint64_t window2,
                    void* workspace, size_t workspace_bytes,
                    uint64_t* cand, uint64_t cap, uint64_t* counters,
                    void* stream);

/* As rfr_stage_match, with bucket regions sized exactly by a count pass over
 * both halves (never overflows; one more enumeration pass). */
int rfr_stage_match_exact(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                          const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                          uint64_t window, uint64_t window2,
                          void* workspace, size_t workspace_bytes,
                          uint64_t* cand, uint64_t cap, uint64_t* counters,
                          void* stream);

/* As rfr_stage_match, always with the fused match that keeps no key tables
 * in device memory: sorted lists of the halves' exact low-subset sums are
 * built by merging, and each CTA generates a range of half a's keys into a
 * shared-memory table and looks half b's keys of that range up in it.
 * rfr_stage_match uses it by itself for 14 <= n_a <= n_b <= 32.  Returns
 * RFR_E_WINDOW if a half has more than 32 elements or the window is too wide
 * for it (about W >= 2^(60 - max(n_a - 14, 2) - 4)); counters[4] = 1 when one
 * key range holds more than 24576 keys of half a (clustered keys), or when
 * the workspace has no room for all fingerprint hits (very wide windows;
 * every hit takes 8 bytes beyond rfr_stage_match_fused_workspace, which has
 * room for 2^20): use rfr_stage_match_exact, or pass more workspace.  The
 * workspace may be rfr_stage_match_fused_workspace(n_a, n_b) bytes (the
 * fused match's own buffers) instead of rfr_stage_match_workspace.
 * Section 3.3. */
int rfr_stage_match_fused(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                          const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                          uint64_t window, uint64_t window2,
                          void* workspace, size_t workspace_bytes,
                          uint64_t* cand, uint64_t cap, uint64_t* counters,
                          void* stream);

/* Match without any allocation (the paper has no counterpart; this is a
 * service for callers that cannot allocate device memory, e.g. inside a host
 * framework that owns all device memory, or a loop where a cudaMalloc that
 * may synchronise the device is not allowed).  Same arguments and results as
 * rfr_stage_match, minus the workspace: it uses a fixed array of
 * RFR_NOALLOC_SCRATCH_BYTES in device memory that every GPU loading the
 * library holds until the process exits.  Halves too large for it are
 * rejected with RFR_E_BUDGET before anything runs (the limit is about
 * n_a, n_b <= 18).  The array's device address is looked up on the first
 * call made with a device current; make that first call before any stream
 * capture.  All calls on a device share the array: calls that overlap on
 * the GPU race and must be serialised by the caller.  The parts of the array
 * that must start at zero are cleared by every call.  The address is cached
 * for the life of the process: after a cudaDeviceReset of that device the
 * cached address is stale, so do not call this entry point on a device that
 * has been reset. */
#define RFR_NOALLOC_SCRATCH_BYTES (16u << 20)
int rfr_stage_match_noalloc(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                            const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                            uint64_t window, uint64_t window2,
                            uint64_t* cand, uint64_t cap, uint64_t* counters,
                            void* stream);

/* K-f verify.  For job j: problem prob[j], element pattern
 * (pat_lo[j], pat_hi[j]) over that problem's n elements.  Builds the real
 * factor of Eq. 2 for the pattern or its complement (whichever has the
 * lower degree) in double-double arithmetic, rounds it, and divides p by it
 * exactly in 128-bit integers.  result[j] = 1 if the pattern's polynomial is
 * an integer divisor of p, 0 if not, RFR_E_OVERFLOW if the test needed more
 * than the integer range; if coeffs_out is not NULL and result[j] == 1, the
 * pattern's own polynomial (degree = sum of element degrees) is written to
 * coeffs_out[j*RFR_LDC ...] ascending.  FACTOR, Section 2. */
int rfr_stage_verify(const int64_t* coeffs, const int32_t* degrees,
                     const double* roots, const rfr_plan* plans,
                     const int32_t* prob, const uint64_t* pat_lo,
                     const uint64_t* pat_hi, int jobs,
                     int32_t* result, int64_t* coeffs_out, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* RFR_STAGES_H_ */
