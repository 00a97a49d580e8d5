// k_splat.cu — the paper's own GPU match (Section 4, Algorithm E): half b is
// splat-sorted (Algorithm D's SPLAT with the atomic-exchange INSERT of
// Section 4) into an array of 2^(n_b+1) home cells (c = 2), and every
// pattern of half a queries it for the sums in its circular window.
//
// A cell holds e(s) = ((S_b(s) >> 1) & ~(2^n_b - 1)) | s for the pattern s of
// half b and its sum S_b(s) = sum_{j in s} w_b[j] (mod 2^64); empty cells hold
// ~0.  e < 2^63, its home cell is e >> (62 - n_b) (= floor(2^(n_b+1) x) for
// x = e / 2^63), and e is non-decreasing in S_b, so the splat array is
// sorted by S_b up to the 2^(n_b+1) units the encoding drops.
//
// INSERT: a thread exchanges its value into the home cell; an empty cell
// ends it; a larger value that comes back moves on to the next cell (the
// thread's value stays); a smaller one is put back on the next exchange and
// the thread's value moves on.  Every cell keeps the smallest value that has
// passed it, so the final array is the sequential one, whatever the order
// of the exchanges.  The step to the next cell is linear, into 4096 overflow
// cells past the last home cell, so the array stays sorted in index order.
//
// QUERY (band form): for a pattern s_a of half a with sum S_a, the values S_b
// with dist(S_a + S_b) <= W lie in one or two linear ranges [lo, hi] of
// S_b (two when the window wraps past 0).  Each range is scanned from the
// home cell of its smallest cell value; the scan stops at the first value
// above the range or at the first empty cell at or past the home cell of
// its largest value.  Values in range are re-checked exactly (Tr_1 window W,
// then the Tr_2 window W2) before a candidate s_a | s_b << n_a is written.
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include "k_match.cuh"
#include "rfr_device.cuh"
#include "rfr_stages.h"

namespace rfr {
namespace {

constexpr int SP_THREADS = 256;
constexpr int SP_LOG = 11;                  // patterns per CTA: 2^SP_LOG (the low bits of the mask)
constexpr uint64_t SP_EMPTY = ~0ull;
constexpr int SP_MAX_STEPS = 4096;          // cells one insertion may move over
constexpr int SP_MAX_XCHG = 4 * SP_MAX_STEPS;
constexpr int SP_MAX_N = 30;

struct SplatJob {
    const uint64_t* w_a; const uint64_t* w2_a;
    const uint64_t* w_b; const uint64_t* w2_b;
    int n_a, n_b;
    unsigned ins_base, qry_base;            // first CTA of this job in the insert / query grids
    uint64_t W, W2;
    uint64_t* gamma;                        // splat_cells(n_b) cells
    uint64_t* cand;
    uint64_t cap;
    unsigned long long* ctr;                // [8]
};

__host__ __device__ inline uint64_t splat_cells(int n) { return (2ull << n) + SPLAT_TAIL; }
__host__ inline unsigned splat_ctas(int n) { return n > SP_LOG ? 1u << (n - SP_LOG) : 1u; }
__device__ inline uint64_t circ_dist(uint64_t v) { return v < (0ull - v) ? v : 0ull - v; }

__device__ inline int find_job(const SplatJob* jobs, int nj, bool ins) {
    int lo = 0, hi = nj - 1;
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if ((ins ? jobs[mid].ins_base : jobs[mid].qry_base) <= blockIdx.x) lo = mid;
        else hi = mid - 1;
    }
    return lo;
}

__device__ inline void warp_add(unsigned long long* dst, unsigned v) {
    v = __reduce_add_sync(0xffffffffu, v);
    if ((threadIdx.x & 31) == 0 && v) atomicAdd(dst, (unsigned long long)v);
}

// SPLAT of half b.  ctr[4] <- 1 if an insertion ran past the overflow tail
// or past its step limit (the array then misses values); ctr[5] += cells
// looked at (Theorem 3.4.2's C times 2^n_b); ctr[6] += atomic exchanges.
__global__ void __launch_bounds__(SP_THREADS) k_splat_insert(const SplatJob* __restrict__ jobs, int nj) {
    __shared__ int s_job;
    __shared__ uint64_t s_w[32];
    __shared__ uint64_t s_hi;
    if (threadIdx.x == 0) s_job = find_job(jobs, nj, true);
    __syncthreads();
    const SplatJob& J = jobs[s_job];
    const int n = J.n_b;
    const int L = n < SP_LOG ? n : SP_LOG;
    const uint64_t hix = blockIdx.x - J.ins_base;
    if (threadIdx.x < n) s_w[threadIdx.x] = J.w_b[threadIdx.x];
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t h = 0;
        for (int b = 0; b < n - L; ++b)
            if ((hix >> b) & 1) h += s_w[L + b];
        s_hi = h;
    }
    __syncthreads();
    const uint64_t lm = (1ull << n) - 1;
    const int hs = 62 - n;
    const uint64_t ncell = splat_cells(n);
    unsigned long long* gamma = (unsigned long long*)J.gamma;
    unsigned visited = 0, xchg = 0;
    bool err = false;
    for (int j = threadIdx.x; j < (1 << L); j += SP_THREADS) {
        uint64_t S = s_hi;
        for (int b = 0; b < L; ++b)
            if ((j >> b) & 1) S += s_w[b];
        unsigned long long x = ((S >> 1) & ~lm) | (hix << L) | (uint64_t)j;
        uint64_t i = x >> hs;
        int steps = 0, ex = 0;
        for (;;) {
            const unsigned long long y = atomicExch(gamma + i, x);
            ++ex;
            if (y == SP_EMPTY) break;
            if (y > x) {                       // x stays here; y moves on
                ++i; ++steps;
                if (i >= ncell || steps >= SP_MAX_STEPS) { err = true; break; }
            }
            x = y;                             // y < x: put y back on the next exchange, x comes back
            if (ex >= SP_MAX_XCHG) { err = true; break; }
        }
        visited += (unsigned)steps + 1;
        xchg += (unsigned)ex;
    }
    warp_add(&J.ctr[5], visited);
    warp_add(&J.ctr[6], xchg);
    if (err) atomicExch(&J.ctr[4], 1ull);
}

// QUERY from every pattern of half a.  ctr[0] += cells in a scanned range
// (coarse), ctr[1] += pairs within W, ctr[2] += candidates (also within W2,
// not the empty pair), ctr[3] <- 1 when the empty pair is met, ctr[7] += cells
// read.
__global__ void __launch_bounds__(SP_THREADS) k_splat_query(const SplatJob* __restrict__ jobs, int nj) {
    __shared__ int s_job;
    __shared__ uint64_t s_wa[32], s_w2a[32], s_wb[32], s_w2b[32];
    __shared__ uint64_t s_hi, s_hi2;
    if (threadIdx.x == 0) s_job = find_job(jobs, nj, false);
    __syncthreads();
    const SplatJob& J = jobs[s_job];
    const int na = J.n_a, nb = J.n_b;
    const int L = na < SP_LOG ? na : SP_LOG;
    const uint64_t hix = blockIdx.x - J.qry_base;
    if (threadIdx.x < na) { s_wa[threadIdx.x] = J.w_a[threadIdx.x]; s_w2a[threadIdx.x] = J.w2_a[threadIdx.x]; }
    if (threadIdx.x < nb) { s_wb[threadIdx.x] = J.w_b[threadIdx.x]; s_w2b[threadIdx.x] = J.w2_b[threadIdx.x]; }
    __syncthreads();
    if (threadIdx.x == 0) {
        uint64_t h = 0, h2 = 0;
        for (int b = 0; b < na - L; ++b)
            if ((hix >> b) & 1) { h += s_wa[L + b]; h2 += s_w2a[L + b]; }
        s_hi = h; s_hi2 = h2;
    }
    __syncthreads();
    const uint64_t lmb = (1ull << nb) - 1;
    const int hs = 62 - nb;
    const uint64_t ncell = splat_cells(nb);
    const uint64_t W = J.W, W2 = J.W2;
    const uint64_t* gamma = J.gamma;
    unsigned coarse = 0, within = 0, reads = 0;
    for (int j = threadIdx.x; j < (1 << L); j += SP_THREADS) {
        const uint64_t sa = (hix << L) | (uint64_t)j;
        uint64_t S = s_hi, S2 = s_hi2;
        for (int b = 0; b < L; ++b)
            if ((j >> b) & 1) { S += s_wa[b]; S2 += s_w2a[b]; }
        const uint64_t t = 0ull - S;                        // S_b near -S_a
        uint64_t lo[2], hi[2];
        int np = 1;
        if (t >= W && t <= ~0ull - W) { lo[0] = t - W; hi[0] = t + W; }
        else { lo[0] = t - W; hi[0] = ~0ull; lo[1] = 0; hi[1] = t + W; np = 2; }
        for (int p = 0; p < np; ++p) {
            const uint64_t eL = (lo[p] >> 1) & ~lmb, eH = ((hi[p] >> 1) & ~lmb) | lmb;
            const uint64_t hH = eH >> hs;
            for (uint64_t i = eL >> hs; i < ncell; ++i) {
                const uint64_t c = __ldg(gamma + i);
                ++reads;
                if (c == SP_EMPTY) {
                    if (i >= hH) break;
                    continue;
                }
                if (c > eH) break;
                if (c < eL) continue;
                ++coarse;
                const uint64_t sb = c & lmb;
                uint64_t Sb = 0, Sb2 = 0;
                for (int b = 0; b < nb; ++b)
                    if ((sb >> b) & 1) { Sb += s_wb[b]; Sb2 += s_w2b[b]; }
                if (circ_dist(S + Sb) > W) continue;
                ++within;
                if (sa == 0 && sb == 0) { atomicExch(&J.ctr[3], 1ull); continue; }
                if (circ_dist(S2 + Sb2) > W2) continue;
                const unsigned long long k = atomicAdd(&J.ctr[2], 1ull);
                if (k < J.cap) J.cand[k] = sa | (sb << na);
            }
        }
    }
    warp_add(&J.ctr[0], coarse);
    warp_add(&J.ctr[1], within);
    warp_add(&J.ctr[7], reads);
}

SplatJob make_job(const ProbJob& p) {
    SplatJob j;
    j.w_a = p.w_a; j.w2_a = p.w2_a; j.w_b = p.w_b; j.w2_b = p.w2_b;
    j.n_a = p.n_a; j.n_b = p.n_b;
    j.ins_base = j.qry_base = 0;
    j.W = p.W; j.W2 = p.W2;
    j.gamma = p.gamma;
    j.cand = p.cand; j.cap = p.cap;
    j.ctr = p.ctr;
    return j;
}

// Fill the gammas, upload the jobs and launch insert then query (queries
// only when `query`).
cudaError_t launch_splat(std::vector<SplatJob>& J, void* dev_jobs, cudaStream_t s, bool query) {
    unsigned ins = 0, qry = 0;
    for (auto& j : J) {
        j.ins_base = ins; ins += splat_ctas(j.n_b);
        j.qry_base = qry; qry += splat_ctas(j.n_a);
        cudaError_t e = cudaMemsetAsync(j.gamma, 0xff, splat_cells(j.n_b) * 8, s);
        if (e != cudaSuccess) return e;
    }
    cudaError_t e = cudaMemcpyAsync(dev_jobs, J.data(), J.size() * sizeof(SplatJob), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    k_splat_insert<<<ins, SP_THREADS, 0, s>>>((const SplatJob*)dev_jobs, (int)J.size());
    if (query) k_splat_query<<<qry, SP_THREADS, 0, s>>>((const SplatJob*)dev_jobs, (int)J.size());
    return cudaGetLastError();
}

}  // namespace

bool splat_geometry(int n_a, int n_b, MatchGeom* g) {
    if (n_a < 0 || n_b < n_a || n_b > SP_MAX_N) return false;
    g->n_a = n_a; g->n_b = n_b;
    g->splat = true;
    g->fused = false;
    g->optimistic = false;
    g->bytes = (splat_cells(n_b) * 8 + 255) & ~(uint64_t)255;
    return true;
}

uint64_t* splat_layout(const MatchGeom& g, char* ws, ProbJob* pj) {
    pj->splat = 1;
    pj->fused = 0;
    pj->n_a = g.n_a; pj->n_b = g.n_b;
    pj->gamma = (uint64_t*)ws;
    return pj->gamma;
}

cudaError_t run_splat(const ProbJob* const* S, int nS, void* dev_jobs, cudaStream_t s) {
    std::vector<SplatJob> J;
    J.reserve(nS);
    for (int i = 0; i < nS; ++i) J.push_back(make_job(*S[i]));
    return launch_splat(J, dev_jobs, s, true);
}

}  // namespace rfr

using namespace rfr;

extern "C" size_t rfr_stage_splat_cells(int n) {
    if (n < 0 || n > SP_MAX_N) return 0;
    return (size_t)splat_cells(n) + 32;               // + 256 bytes for the launch descriptor
}

static int splat_stage(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                       const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                       uint64_t window, uint64_t window2, uint64_t* gamma, size_t gamma_cells,
                       uint64_t* cand, uint64_t cap, unsigned long long* counters, void* stream, bool query) {
    if (n_b < 0 || n_b > SP_MAX_N || (n_b && !w_b) || !gamma || !counters) return RFR_E_INVALID;
    if (query && (n_a < 0 || n_a > n_b || (n_a && (!w_a || !w2_a)) || (n_b && !w2_b) || (cap && !cand)))
        return RFR_E_INVALID;
    if (query && window >= (1ull << 63)) return RFR_E_WINDOW;
    if ((((uintptr_t)gamma) & 255) || gamma_cells < rfr_stage_splat_cells(n_b)) return RFR_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    std::vector<SplatJob> J(1);
    SplatJob& j = J[0];
    j.w_a = w_a; j.w2_a = w2_a; j.w_b = w_b; j.w2_b = w2_b;
    j.n_a = query ? n_a : 0; j.n_b = n_b;
    j.W = window; j.W2 = window2;
    j.gamma = gamma;
    j.cand = cand; j.cap = cap;
    j.ctr = counters;
    if (cudaMemsetAsync(counters, 0, 8 * 8, s) != cudaSuccess) return RFR_E_CUDA;
    void* dj = gamma + splat_cells(n_b);
    if (launch_splat(J, dj, s, query) != cudaSuccess) return RFR_E_CUDA;
    return RFR_OK;
}

extern "C" int rfr_stage_splat(const uint64_t* w, int n, uint64_t* gamma, size_t gamma_cells,
                               unsigned long long* counters, void* stream) {
    return splat_stage(nullptr, nullptr, 0, w, nullptr, n, 0, 0, gamma, gamma_cells, nullptr, 0,
                       counters, stream, false);
}

extern "C" int rfr_stage_splat_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                                     const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                                     uint64_t window, uint64_t window2, uint64_t* gamma, size_t gamma_cells,
                                     uint64_t* cand, uint64_t cap, unsigned long long* counters, void* stream) {
    return splat_stage(w_a, w2_a, n_a, w_b, w2_b, n_b, window, window2, gamma, gamma_cells, cand, cap,
                       counters, stream, true);
}
