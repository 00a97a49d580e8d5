// k_prune.cu — Algorithm B (Section 3.2, RECOMBINE_B) on the GPU: the
// search over all 2^m patterns of the m searched elements, pruned by jumps.
//
// The elements are sorted ascending (w_1 <= ... <= w_m, uint64 fixed point,
// M = 2^64) with prefix sums sigma_i.  After the pattern s with value x, the
// next 2^j - 1 patterns (j at most the trailing zero bits of s) have values
// x + t for the non-empty sums t of the j smallest elements, inside
// [x + w_1, x + sigma_j]; none is accepted (circular window W, Eq. 9) when
// x + w_1 > W and x + sigma_j < M - W, and the search jumps to s + 2^j for
// the largest such j.
//
// The pattern space is cut into aligned blocks of 2^B patterns, one thread
// per block (B = m - 20 for m > 20, so about 2^20 threads per problem); a
// jump never leaves its block.  The value follows the jumps in O(1): adding
// 2^j to s clears the run of ones at bits j .. k-1 and sets bit k, so
// x += w_k - (sigma_k - sigma_j) modulo 2^64.  Accepted patterns other than
// the empty one are checked against the Tr_2 window W2 and written in the
// original element order.
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include "k_match.cuh"
#include "rfr_device.cuh"
#include "rfr_stages.h"

namespace rfr {
namespace {

constexpr int PR_THREADS = 256;
constexpr int PR_BLOCK_LOG = 20;           // at most 2^20 blocks (threads) per problem

struct PruneJob {
    const uint64_t* w; const uint64_t* w2;
    int m, B;                              // searched elements; patterns per thread 2^B
    unsigned cta_base;                     // first CTA of this job in the grid
    uint64_t W, W2;
    uint64_t* cand;
    uint64_t cap;
    unsigned long long* ctr;               // [8]
};

__host__ inline int prune_B(int m) { return m > PR_BLOCK_LOG ? m - PR_BLOCK_LOG : 0; }
__host__ inline unsigned prune_ctas(int m) {
    const uint64_t th = 1ull << (m - prune_B(m));
    return (unsigned)((th + PR_THREADS - 1) / PR_THREADS);
}
__device__ inline uint64_t circ_dist(uint64_t v) { return v < (0ull - v) ? v : 0ull - v; }

// ctr[0] += patterns visited, ctr[1] += patterns within W (the empty one
// included), ctr[2] += candidates (also within W2, not empty), ctr[3] <- 1
// when the empty pattern is met.
__global__ void __launch_bounds__(PR_THREADS) k_prune(const PruneJob* __restrict__ jobs, int nj) {
    __shared__ int s_job;
    __shared__ uint64_t ws[PRUNE_MAX_M + 1], w2s[PRUNE_MAX_M + 1], P[PRUNE_MAX_M + 1], S[PRUNE_MAX_M + 1];
    __shared__ int perm[PRUNE_MAX_M + 1];
    if (threadIdx.x == 0) {
        int lo = 0, hi = nj - 1;
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (jobs[mid].cta_base <= blockIdx.x) lo = mid;
            else hi = mid - 1;
        }
        s_job = lo;
        const PruneJob& J = jobs[lo];
        for (int i = 0; i < J.m; ++i) {                 // insertion sort with the original indices
            const uint64_t v = J.w[i];
            int k = i;
            while (k > 0 && ws[k - 1] > v) { ws[k] = ws[k - 1]; perm[k] = perm[k - 1]; --k; }
            ws[k] = v;
            perm[k] = i;
        }
        P[0] = 0;
        S[0] = 0;
        for (int i = 0; i < J.m; ++i) {
            w2s[i] = J.w2[perm[i]];
            P[i + 1] = P[i] + ws[i];                                    // modulo 2^64
            S[i + 1] = S[i] > ~0ull - ws[i] ? ~0ull : S[i] + ws[i];     // as integers, saturated
        }
        ws[J.m] = 0;
    }
    __syncthreads();
    const PruneJob& J = jobs[s_job];
    const int m = J.m, B = J.B;
    const uint64_t nblk = 1ull << (m - B);
    const uint64_t blk = (uint64_t)(blockIdx.x - J.cta_base) * PR_THREADS + threadIdx.x;
    unsigned steps = 0, within = 0;
    if (blk < nblk) {
        const uint64_t W = J.W;
        const uint64_t w1 = m ? ws[0] : ~0ull;
        uint64_t s = blk << B;
        const uint64_t end = s + (1ull << B);
        uint64_t x = 0;
        for (int i = B; i < m; ++i)
            if ((s >> i) & 1) x += ws[i];
        for (;;) {
            ++steps;
            if (circ_dist(x) <= W) {
                ++within;
                if (s == 0) {
                    atomicExch(&J.ctr[3], 1ull);
                } else {
                    uint64_t t2 = 0, orig = 0;
                    for (int i = 0; i < m; ++i)
                        if ((s >> i) & 1) { t2 += w2s[i]; orig |= 1ull << perm[i]; }
                    if (circ_dist(t2) <= J.W2) {
                        const unsigned long long k = atomicAdd(&J.ctr[2], 1ull);
                        if (k < J.cap) J.cand[k] = orig;
                    }
                }
            }
            int c = s ? __ffsll((long long)s) - 1 : 64;
            if (c > B) c = B;
            int j = 0;
            // values of the skipped patterns lie in [x + w_1, x + sigma_j]
            if (x > W || w1 > W - x) {
                if (x <= ~0ull - W) {
                    const uint64_t lim = ~0ull - W - x;                 // M - W - x - 1
                    while (j < c && S[j + 1] != ~0ull && S[j + 1] <= lim) ++j;
                }
            }
            const uint64_t s2 = s + (1ull << j);
            if (s2 >= end) break;
            const int k = j + __ffsll((long long)~(s >> j)) - 1;       // lowest zero bit of s at or above j
            x = x - (P[k] - P[j]) + ws[k];
            s = s2;
        }
    }
    steps = __reduce_add_sync(0xffffffffu, steps);
    within = __reduce_add_sync(0xffffffffu, within);
    if ((threadIdx.x & 31) == 0) {
        if (steps) atomicAdd(&J.ctr[0], (unsigned long long)steps);
        if (within) atomicAdd(&J.ctr[1], (unsigned long long)within);
    }
}

cudaError_t launch_prune(std::vector<PruneJob>& J, void* dev_jobs, cudaStream_t s) {
    unsigned ctas = 0;
    for (auto& j : J) {
        j.B = prune_B(j.m);
        j.cta_base = ctas;
        ctas += prune_ctas(j.m);
    }
    cudaError_t e = cudaMemcpyAsync(dev_jobs, J.data(), J.size() * sizeof(PruneJob), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_prune<<<ctas, PR_THREADS, 0, s>>>((const PruneJob*)dev_jobs, (int)J.size());
    return cudaGetLastError();
}

}  // namespace

bool prune_geometry(int n_a, int n_b, MatchGeom* g) {
    if (n_a < 0 || n_b < 0 || n_a + n_b > PRUNE_RUNTIME_MAX_M) return false;
    g->n_a = n_a; g->n_b = n_b;
    g->prune = true;
    g->splat = false;
    g->fused = false;
    g->optimistic = false;
    g->bytes = 256;
    return true;
}

cudaError_t run_prune(const ProbJob* const* Pj, int nP, void* dev_jobs, cudaStream_t s) {
    std::vector<PruneJob> J(nP);
    for (int i = 0; i < nP; ++i) {
        const ProbJob& p = *Pj[i];
        PruneJob& j = J[i];
        j.w = p.w_a; j.w2 = p.w2_a;                      // the searched elements are contiguous
        j.m = p.n_a + p.n_b;
        j.W = p.W; j.W2 = p.W2;
        j.cand = p.cand; j.cap = p.cap;
        j.ctr = p.ctr;
    }
    return launch_prune(J, dev_jobs, s);
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_prune(const uint64_t* w, const uint64_t* w2, int m, uint64_t window, uint64_t window2,
                               uint64_t* cand, uint64_t cap, unsigned long long* counters,
                               void* workspace, size_t workspace_bytes, void* stream) {
    if (m < 0 || m > PRUNE_MAX_M || (m && (!w || !w2)) || !counters || (cap && !cand)) return RFR_E_INVALID;
    if (!workspace || workspace_bytes < 256 || (((uintptr_t)workspace) & 255)) return RFR_E_INVALID;
    if (window >= (1ull << 63)) return RFR_E_WINDOW;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<PruneJob> J(1);
    J[0].w = w; J[0].w2 = w2; J[0].m = m;
    J[0].W = window; J[0].W2 = window2;
    J[0].cand = cand; J[0].cap = cap;
    J[0].ctr = counters;
    if (cudaMemsetAsync(counters, 0, 8 * 8, s) != cudaSuccess) return RFR_E_CUDA;
    return launch_prune(J, workspace, s) == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
