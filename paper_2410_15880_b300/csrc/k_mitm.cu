// k_mitm.cu — fused meet-in-the-middle match (K-c + K-d + K-e of Section 3.3
// for large halves, with no key tables in device memory).
//
// Each half's h elements are split into low elements 0..l-1 and high
// elements l..h-1.  The sorted list Y of all 2^l low-subset sums is built
// once per half by merging (k_ybuild_smem, k_ymerge: the sorted list of a
// set plus one element is the merge of the list and its copy shifted by the
// element's weight).  The low weights are rounded to multiples of 2^l for
// the list, so an entry is its sum's high bits with the subset's mask below.  Every high subset x gives one sorted run x + Y
// (rotated to start at its smallest key), so a half is 2^(h-l) sorted runs.
//
// The key space [0, 2^64) is cut into 2^d1 units of width U.  One CTA walks a
// slab of consecutive units and keeps one cursor per run; per unit it
//   1. reads, from every run of half a, the stretch of keys inside the unit
//      and appends them, as 16-bit fingerprints of their position in the
//      unit plus their pattern masks, to a shared-memory table with one
//      linked list per bin, marking each key's cell in an occupancy bitmap;
//   2. reads, from every run of half b, the stretch of keys within Wc of the
//      unit, [lo - Wc, hi + Wc) (circularly), tests the one or two bitmap
//      cells its window touches and, for the few keys whose cells are
//      occupied, walks the lists of the bins around it (queued per warp and
//      walked 32 at a time, so that lanes do not wait on each other).
// A pair (a, b) with |K_a - K_b| < Wc (keys of half b are negated sums, so
// K_a - K_b is the pattern's Tr_1 value) is met exactly once, in the unit
// holding K_a.  Fingerprint hits are re-checked exactly against the Tr_1
// window W (Eq. 9 / Eq. 19, circular) and the Tr_2 window W2, as in the table
// join, so the candidate set is the same as RECOMBINE_C's.
#include <algorithm>
#include <cstdint>
#include <cstring>
#include <vector>
#include <cuda_runtime.h>
#include "k_match.cuh"
#include "rfr_device.cuh"
#include "rfr_stages.h"

namespace rfr {
namespace {

constexpr int YS_LOG = 12;                                     // list levels built in shared memory
constexpr int YS_THREADS = 1024;
constexpr size_t YS_SMEM = ((size_t)2 << YS_LOG) * 8;          // two buffers of 2^12 entries
constexpr int YM_THREADS = 256;
constexpr int YM_PER = 8;                                      // merge outputs per thread (2048-output tiles: 32 KB of shared memory, 7 CTAs per SM)

constexpr int MT_THREADS = 1024;
constexpr int MT_ACAP = 12288;                                 // table-a keys of one unit (mean 8192)
constexpr int MT_POOL = MT_ACAP / 8;                           // shared slots for warps that fill their own
constexpr int MT_NBL = 12;                                     // at most 2^12 bins per unit
constexpr int MT_RUNS = 1024;                                  // runs per half
constexpr int MT_BM_LOG = 19;                                  // occupancy bitmap: about 2^19 cells per unit
constexpr int MT_BMW = (1 << (MT_BM_LOG - 5)) + 4;             // + margin cells on both sides (16-byte multiple)
constexpr int MT_QCAP = 64;                                    // deferred lookups per warp
constexpr int GL = 8;                                          // lanes walking one run together
constexpr uint32_t MT_NIL = 0xffffffffu;
constexpr size_t MT_SMEM = (size_t)MT_ACAP * (4 + 2 + 2) + ((size_t)4 << MT_NBL) + (size_t)MT_BMW * 4 +
                           (size_t)MT_RUNS * (8 + 4 + 4) * 2 + (size_t)(MT_THREADS / 32) * MT_QCAP * 8;

__device__ __forceinline__ uint64_t mt_lowmask(int h) { return h ? (~0ull >> (64 - h)) : 0ull; }

__device__ __forceinline__ uint32_t lower_bound_keys(const uint64_t* K, uint32_t n, uint64_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (K[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Outputs d0 .. d1-1 of the merge of the sorted entries K[0..n) with the sorted
// sequence B[t] = K[(r + t) mod n] + c (K shifted by c, rotated to its smallest
// element; equal entries take K first).  n is a power of two.
template <class Out>
__device__ __forceinline__ void merge_range(const uint64_t* __restrict__ K, uint32_t n, uint32_t r, uint64_t c,
                                            uint32_t d0, uint32_t d1, Out out) {
    const uint32_t nm = n - 1;
    uint32_t lo = d0 > n ? d0 - n : 0, hi = d0 < n ? d0 : n;
    while (lo < hi) {                                          // merge path: K's share of the first d0
        const uint32_t mid = (lo + hi) >> 1;
        if (K[mid] <= K[(r + d0 - mid - 1) & nm] + c) lo = mid + 1; else hi = mid;
    }
    uint32_t a = lo, b = d0 - lo;
    for (uint32_t d = d0; d < d1; ++d) {
        const uint64_t ka = a < n ? K[a] : 0ull;
        const uint64_t kb = b < n ? K[(r + b) & nm] + c : 0ull;
        if (b >= n || (a < n && ka <= kb)) { out(d, ka); ++a; }
        else { out(d, kb); ++b; }
    }
}

// List entries are (S & ~(2^l - 1)) | mask, where S is the sum over the mask of
// the low weights rounded to multiples of 2^l (so |S - exact sum| <= l * 2^(l-1)).
// Adding element i to every entry is adding the constant c_i = round(w_i) + 2^i:
// the mask bits never carry into S.
__device__ __forceinline__ uint64_t list_step(const uint64_t* w, int neg, int i, int l) {
    const uint64_t wi = neg ? 0ull - w[i] : w[i];
    const uint64_t half = l ? 1ull << (l - 1) : 0ull;
    return ((wi + half) & ~mt_lowmask(l)) + (1ull << i);
}

struct YJob {
    const uint64_t* w;          // the half's weights (elements 0..l-1 used)
    int l, neg;                 // list bits; keys are negated sums for half b
    uint64_t* kb[2];            // [2^(l-1)] intermediate levels, ping-pong (l > YS_LOG only)
    uint64_t* ylist;            // [2^l] result, ascending
    uint32_t* splits;           // [2^l / YM_TILE + 2]: a level's tile starts on the merge path, then its rotation
};

// Levels 0 .. min(l, 12) - 1 of one half's list in shared memory.
__global__ void __launch_bounds__(YS_THREADS) k_ybuild_smem(const YJob* __restrict__ js) {
    extern __shared__ __align__(16) uint64_t ys_sm[];
    uint64_t* Kb[2] = {ys_sm, ys_sm + (1 << YS_LOG)};
    const YJob J = js[blockIdx.x];
    const int s = J.l < YS_LOG ? J.l : YS_LOG;
    if (threadIdx.x == 0) Kb[0][0] = 0ull;
    __syncthreads();
    for (int i = 0; i < s; ++i) {
        const uint32_t n = 1u << i;
        const uint64_t c = list_step(J.w, J.neg, i, J.l);
        const uint64_t* K = Kb[i & 1];
        uint64_t* KO = Kb[(i + 1) & 1];
        const uint32_t r = lower_bound_keys(K, n, 0ull - c);   // first entry that wraps when c is added
        const uint32_t tot = 2 * n, per = (tot + blockDim.x - 1) / blockDim.x;
        const uint32_t d0 = min(tot, threadIdx.x * per), d1 = min(tot, d0 + per);
        if (d0 < d1) merge_range(K, n, r, c, d0, d1, [&](uint32_t d, uint64_t k) { KO[d] = k; });
        __syncthreads();
    }
    const uint64_t* K = Kb[s & 1];
    uint64_t* out = s == J.l ? J.ylist : J.kb[0];
    for (uint32_t j = threadIdx.x; j < (1u << s); j += blockDim.x) out[j] = K[j];
}

// Level i >= 12 (2^i entries -> 2^(i+1)) for every half with l > i; cpl CTAs per
// half, each writing a tile of YM_TILE outputs.  The CTA finds where its tile
// starts and ends on the merge path (two binary searches over the list), reads
// the two input stretches into shared memory with coalesced loads, merges them
// there (YM_PER outputs per thread) and writes the tile back coalesced.  The
// last level writes the list itself.
constexpr int YM_TILE = YM_THREADS * YM_PER;
constexpr size_t YM_SMEM = (size_t)2 * YM_TILE * 8;

__device__ __forceinline__ uint32_t merge_split(const uint64_t* __restrict__ K, uint32_t n, uint32_t r,
                                                uint64_t c, uint32_t d) {
    const uint32_t nm = n - 1;
    uint32_t lo = d > n ? d - n : 0, hi = d < n ? d : n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (K[mid] <= K[(r + d - mid - 1) & nm] + c) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// Tile boundaries of level i: thread (half h, boundary c) finds how many of the
// first c * YM_TILE merged entries come from the list itself (merge path), and
// boundary 0 also stores the rotation of the shifted copy.
__global__ void __launch_bounds__(128) k_ysplit(const YJob* __restrict__ js, int nh, int i, int cpl) {
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= nh * (cpl + 1)) return;
    const YJob& J = js[t / (cpl + 1)];
    const int c = t % (cpl + 1);
    const uint32_t n = 1u << i;
    const uint64_t* __restrict__ K = J.kb[(i - YS_LOG) & 1];
    const uint64_t cs = list_step(J.w, J.neg, i, J.l);
    const uint32_t r = lower_bound_keys(K, n, 0ull - cs);
    J.splits[c] = merge_split(K, n, r, cs, (uint32_t)c * YM_TILE);
    if (c == 0) J.splits[cpl + 1] = r;
}

__global__ void __launch_bounds__(YM_THREADS) k_ymerge(const YJob* __restrict__ js, int i, int cpl) {
    extern __shared__ __align__(16) uint64_t ym_sm[];
    uint64_t* tin = ym_sm;                        // [YM_TILE]: the stretch of K, then of the shifted copy
    uint64_t* tout = ym_sm + YM_TILE;             // [YM_TILE]: merged tile
    const YJob& J = js[blockIdx.x / cpl];
    const int c = blockIdx.x % cpl;
    const uint32_t n = 1u << i, nm = n - 1;
    const int p = (i - YS_LOG) & 1;
    const uint64_t* __restrict__ K = J.kb[p];
    const uint64_t cs = list_step(J.w, J.neg, i, J.l);
    const uint32_t r = J.splits[cpl + 1];
    const uint32_t o0 = (uint32_t)c * YM_TILE;
    const uint32_t a0 = J.splits[c], a1 = J.splits[c + 1], b0 = o0 - a0;
    const uint32_t na = a1 - a0;                  // nb = YM_TILE - na
    for (uint32_t j = threadIdx.x; j < (uint32_t)YM_TILE; j += blockDim.x)
        tin[j] = j < na ? K[a0 + j] : K[(r + b0 + (j - na)) & nm] + cs;
    __syncthreads();
    // local merge of tin[0..na) with tin[na..YM_TILE)
    const uint32_t nb = YM_TILE - na, dl = threadIdx.x * YM_PER;
    const uint64_t* A = tin;
    const uint64_t* Bv = tin + na;
    uint32_t lo = dl > nb ? dl - nb : 0, hi = dl < na ? dl : na;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (A[mid] <= Bv[dl - mid - 1]) lo = mid + 1; else hi = mid;
    }
    uint32_t ia = lo, ib = dl - lo;
    for (int q = 0; q < YM_PER; ++q) {
        const uint64_t ka = ia < na ? A[ia] : ~0ull;
        const uint64_t kb = ib < nb ? Bv[ib] : ~0ull;
        const bool ta = ib >= nb || (ia < na && ka <= kb);
        tout[dl + q] = ta ? ka : kb;
        if (ta) ++ia; else ++ib;
    }
    __syncthreads();
    uint64_t* KO = i == J.l - 1 ? J.ylist : J.kb[p ^ 1];
    for (uint32_t j = threadIdx.x; j < (uint32_t)YM_TILE; j += blockDim.x) KO[o0 + j] = tout[j];
}

struct MitmJob {
    const uint64_t* ya;  const uint64_t* yb;                 // sorted low lists
    const uint64_t* w_a; const uint64_t* w2_a;
    const uint64_t* w_b; const uint64_t* w2_b;
    int n_a, n_b, l_a, l_b;
    int d1, nbl, slab, wf;                                    // units, bins per unit, units per CTA, fingerprint window
    int cta_base, c_lo;                                       // first CTA in the grid; first slab (key-range shard)
    uint64_t W, W2, Wc;
    uint64_t* cand;
    uint64_t cap;
    unsigned long long* ctr;
    int* err;
    uint64_t* hits;                                           // fingerprint hits: ma | mb << 32
    unsigned long long* nhits;
    uint64_t hcap;
};

__device__ __forceinline__ uint64_t mask_sum(const uint64_t* w, uint32_t m) {
    uint64_t s = 0;
    for (; m; m &= m - 1) s += w[__ffs(m) - 1];
    return s;
}

// First rotated index t in [0, N] of run (x, j0) with key >= v (keys rise along t).
__device__ __forceinline__ uint32_t run_lower_bound(const uint64_t* Y, uint32_t j0, uint32_t N, uint64_t x,
                                                    uint64_t keep, uint64_t v) {
    uint32_t lo = 0, hi = N;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (x + (Y[(j0 + mid) & (N - 1)] & keep) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// First index j of the (unrotated) list with (Y[j] & keep) >= v.
__device__ __forceinline__ uint32_t list_lower_bound(const uint64_t* Y, uint32_t N, uint64_t keep, uint64_t v) {
    uint32_t lo = 0, hi = N;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if ((Y[mid] & keep) < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

__global__ void __launch_bounds__(MT_THREADS, 1) k_mitm(const MitmJob* __restrict__ js, int np) {
    extern __shared__ __align__(16) unsigned char mt_sm[];
    uint32_t* msk = reinterpret_cast<uint32_t*>(mt_sm);                // [ACAP] table-a masks
    uint32_t* head = msk + MT_ACAP;                                     // [bins] first key of each bin (list)
    uint32_t* bm = head + (1 << MT_NBL);                                // [BMW] cells holding a table-a key
    uint64_t* xa = reinterpret_cast<uint64_t*>(bm + MT_BMW);            // run offsets, half a
    uint64_t* xb = xa + MT_RUNS;                                        // run offsets, half b
    uint2* queue = reinterpret_cast<uint2*>(xb + MT_RUNS);              // [warps][QCAP] deferred lookups
    uint32_t* j0a = reinterpret_cast<uint32_t*>(queue + (MT_THREADS / 32) * MT_QCAP);
    uint32_t* ta = j0a + MT_RUNS;
    uint32_t* j0b = ta + MT_RUNS;
    uint32_t* tb = j0b + MT_RUNS;
    uint16_t* fpr = reinterpret_cast<uint16_t*>(tb + MT_RUNS);          // [ACAP] table-a fingerprints
    uint16_t* nxt = fpr + MT_ACAP;                                      // [ACAP] next key of the same bin
    __shared__ uint64_t wa[32], wb[32];
    __shared__ uint32_t s_count;

    int jl = 0, jh = np - 1;                                            // last job with cta_base <= blockIdx.x
    while (jl < jh) {
        const int mid = (jl + jh + 1) >> 1;
        if (js[mid].cta_base <= (int)blockIdx.x) jl = mid; else jh = mid - 1;
    }
    const MitmJob& P = js[jl];
    const int c = blockIdx.x - P.cta_base + P.c_lo;
    const int n_a = P.n_a, n_b = P.n_b, la = P.l_a, lb = P.l_b;
    const uint32_t Na = 1u << la, Nb = 1u << lb;
    const int RA = 1 << (n_a - la), RB = 1 << (n_b - lb);
    const uint64_t keepa = ~mt_lowmask(la), keepb = ~mt_lowmask(lb);
    const int d1 = P.d1, su = 64 - d1, nbl = P.nbl, bsh = su - nbl, fsh = bsh - 16;
    const uint32_t NB = 1u << d1;
    const uint64_t U = 1ull << su;
    const uint64_t Wc = P.Wc;
    const int wf = P.wf;
    const int nbins = 1 << nbl;
    // cells of 2^rsh fingerprint positions, wider than 2 wf, shifted by one cell so
    // that the windows of keys just outside the unit stay at cell >= 0
    int rsh = nbl + 16 > MT_BM_LOG ? nbl + 16 - MT_BM_LOG : 0;
    while ((1 << rsh) <= 2 * wf + 1) ++rsh;
    const int coff = 1 << rsh;
    const int nbmw = (((1 << (nbl + 16)) >> rsh) + 3 + 31) >> 5;
    const uint64_t* __restrict__ Ya = P.ya;
    const uint64_t* __restrict__ Yb = P.yb;
    const uint32_t k0 = (uint32_t)c * (uint32_t)P.slab, k1 = k0 + (uint32_t)P.slab;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int gi = lane / GL, gl = lane % GL, gsh = gi * GL;          // run group of this lane
    const int gid = warp * (32 / GL) + gi, NG = (int)blockDim.x / GL;
    const uint32_t gbits = (1u << GL) - 1u;
    const uint32_t lma = Na - 1u, lmb = Nb - 1u;                      // low-list masks (l <= 21)
    // table slots: the runs of half a share all but MT_POOL slots equally
    const uint32_t gslots = (uint32_t)((MT_ACAP - MT_POOL) / RA);
    uint2* wq = queue + warp * MT_QCAP;

    if (threadIdx.x < n_a) wa[threadIdx.x] = P.w_a[threadIdx.x];
    if (threadIdx.x < n_b) wb[threadIdx.x] = P.w_b[threadIdx.x];
    __syncthreads();
    // run state: offset x, rotation j0 (index of the smallest key), cursor at the slab's first unit
    for (int g = threadIdx.x; g < RA; g += blockDim.x) {
        uint64_t x = 0;
        for (uint32_t t = (uint32_t)g; t; t &= t - 1) x += wa[la + __ffs(t) - 1];
        const uint32_t j0 = list_lower_bound(Ya, Na, keepa, 0ull - x) & (Na - 1);
        xa[g] = x; j0a[g] = j0;
        ta[g] = k0 ? run_lower_bound(Ya, j0, Na, x, keepa, (uint64_t)k0 << su) : 0u;
    }
    for (int g = threadIdx.x; g < RB; g += blockDim.x) {
        uint64_t x = 0;
        for (uint32_t t = (uint32_t)g; t; t &= t - 1) x -= wb[lb + __ffs(t) - 1];
        const uint32_t j0 = list_lower_bound(Yb, Nb, keepb, 0ull - x) & (Nb - 1);
        xb[g] = x; j0b[g] = j0;
        tb[g] = k0 ? run_lower_bound(Yb, j0, Nb, x, keepb, ((uint64_t)k0 << su) - Wc) : 0u;
    }

    // a fingerprint hit: the pair is re-checked exactly by k_mitm_check
    auto hit = [&](uint32_t ma, uint32_t mb) {
        const unsigned long long idx = atomicAdd(P.nhits, 1ull);
        if (idx < P.hcap) P.hits[idx] = (uint64_t)ma | ((uint64_t)mb << 32);
        else atomicExch(P.err, 1);                                   // more hits than room: redo with tables
    };
    // Does the cell of fingerprint position pb (-wf <= pb < 2^(nbl+16) + wf) hold a
    // table-a key within wf?  (Each key marks every cell its window touches.)
    auto maybe = [&](int pb) -> bool {
        const uint32_t q = (uint32_t)(pb + coff) >> rsh;
        return ((bm[q >> 5] >> (q & 31)) & 1u) != 0u;
    };
    // The table-a keys of the bins around pb: fingerprints within wf are re-checked exactly.
    auto scan_bins = [&](int pb, uint32_t mb) {
        const int plo = pb - wf < 0 ? 0 : pb - wf;
        const int phi = pb + wf > (nbins << 16) - 1 ? (nbins << 16) - 1 : pb + wf;
        for (int bin = plo >> 16; bin <= (phi >> 16); ++bin) {
            uint32_t e = head[bin];
            for (int steps = 0; e < (uint32_t)MT_ACAP && steps < MT_ACAP; ++steps) {   // lists end in NIL; bounded anyway
                const int d = ((bin << 16) | (int)fpr[e]) - pb;
                if (d >= -wf && d <= wf) hit(msk[e], mb);
                e = nxt[e] == 0xffffu ? MT_NIL : nxt[e];
            }
        }
    };
    // Warp-uniform: queue the lanes whose lookup may hit; scan 32 queued lookups at a time.
    uint32_t qn = 0;
    auto enqueue = [&](bool need, int pb, uint32_t run_b, uint32_t ylow) {
        const uint32_t qb = __ballot_sync(0xffffffffu, need);
        if (!qb) return;
        if (need) wq[qn + __popc(qb & lt)] = make_uint2((uint32_t)pb, (run_b << lb) | (ylow & lmb));
        qn += __popc(qb);
        if (qn >= 32) {
            __syncwarp();
            const uint2 e = wq[lane];
            const uint2 e2 = lane + 32 < (int)qn ? wq[lane + 32] : make_uint2(0u, 0u);
            __syncwarp();
            if (lane + 32 < (int)qn) wq[lane] = e2;
            qn -= 32;
            scan_bins((int)e.x, e.y);
        }
    };
    auto drain = [&]() {
        if (!qn) return;
        __syncwarp();
        if (lane < (int)qn) {
            const uint2 e = wq[lane];
            scan_bins((int)e.x, e.y);
        }
        qn = 0;
        __syncwarp();
    };
    // one run of half b, from rotated index t while key - base < span (no cursor update)
    auto walk_b = [&](int g, uint32_t t, uint64_t base, uint64_t span, uint64_t lo) {
        const uint64_t xbb = xb[g] - base, lob = lo - base;
        const uint32_t j0 = j0b[g];
        for (;;) {
            const uint32_t idx = t + lane;
            const uint64_t y = idx < Nb ? Yb[(j0 + idx) & (Nb - 1)] : 0ull;
            const uint64_t rk = xbb + (y & keepb);
            const bool in = idx < Nb && rk < span;
            const int pb = (int)((long long)(rk - lob) >> fsh);
            enqueue(in && maybe(pb), pb, (uint32_t)g, (uint32_t)y);
            const uint32_t cnt = __popc(__ballot_sync(0xffffffffu, in));
            t += cnt;
            if (cnt < 32) break;
        }
    };

    for (uint32_t k = k0; k < k1; ++k) {
        const uint64_t lo = (uint64_t)k << su;
        {   // reset the table heads and the bitmap with 16-byte stores
            uint4* h4 = reinterpret_cast<uint4*>(head);
            for (int b = threadIdx.x; b < (nbins >> 2); b += blockDim.x) h4[b] = make_uint4(MT_NIL, MT_NIL, MT_NIL, MT_NIL);
            uint4* b4 = reinterpret_cast<uint4*>(bm);
            for (int b = threadIdx.x; b < ((nbmw + 3) >> 2); b += blockDim.x) b4[b] = make_uint4(0u, 0u, 0u, 0u);
        }
        if (threadIdx.x == 0) s_count = 0u;
        __syncthreads();
        // ---- table a: every key of the unit.  Groups of GL lanes walk one run each
        // (GL consecutive keys per step, a ring of four chunks in flight); the warp
        // steps until its groups' runs leave the unit.
        {
            for (int run = gid; run - gi < RA; run += NG) {
                bool act = run < RA;
                const int rr = act ? run : 0;
                const uint64_t xl = xa[rr] - lo;
                const uint32_t jj = j0a[rr];
                uint32_t t = act ? ta[rr] : 0u;
                const uint32_t tfirst = t;
                // this run's slots: gslots from gbase (one region per run, so a group that walks
                // several runs in turn keeps all their keys); keys beyond them go to the shared pool
                const uint32_t gbase = MT_POOL + (uint32_t)(act ? run : 0) * gslots;
                // chunks are read unconditionally: the index is taken modulo Na
                uint64_t y0 = Ya[(jj + t + gl) & lma], y1 = Ya[(jj + t + GL + gl) & lma];
                uint64_t y2 = Ya[(jj + t + 2 * GL + gl) & lma], y3 = Ya[(jj + t + 3 * GL + gl) & lma];
                auto step = [&](uint64_t& y) {
                    const uint64_t rel = xl + (y & ~(uint64_t)lma);
                    const bool in = act && t + gl < Na && rel < U;
                    const uint32_t bal = __ballot_sync(0xffffffffu, in);
                    const uint32_t cnt = __popc((bal >> gsh) & gbits);
                    const uint32_t off = t - tfirst + gl;                  // this key's place in the run's stretch
                    uint32_t slot = gbase + off;
                    const uint32_t spill = __ballot_sync(0xffffffffu, in && off >= gslots);
                    if (spill) {                                          // rare: the run overran its slots
                        uint32_t pbase = 0;
                        if (lane == 0) pbase = atomicAdd(&s_count, (uint32_t)__popc(spill));
                        pbase = __shfl_sync(0xffffffffu, pbase, 0) + __popc(spill & lt);
                        if (in && off >= gslots) slot = pbase < (uint32_t)MT_POOL ? pbase : (uint32_t)MT_ACAP;
                    }
                    if (in && slot < (uint32_t)MT_ACAP) {
                        const uint32_t pv = (uint32_t)(rel >> fsh);
                        fpr[slot] = (uint16_t)pv;
                        msk[slot] = ((uint32_t)run << la) | ((uint32_t)y & lma);
                        nxt[slot] = (uint16_t)atomicExch(&head[pv >> 16], slot);
                        const uint32_t q0 = (pv + (uint32_t)(coff - wf)) >> rsh, q1 = (pv + (uint32_t)(coff + wf)) >> rsh;
                        atomicOr(&bm[q0 >> 5], 1u << (q0 & 31));
                        if (q1 != q0) atomicOr(&bm[q1 >> 5], 1u << (q1 & 31));
                    }
                    t += cnt;
                    act = act && cnt == (uint32_t)GL;
                    y = Ya[(jj + t + 3 * GL + gl) & lma];                 // the chunk four ahead
                };
                for (;;) {
                    if (!__any_sync(0xffffffffu, act)) break;
                    step(y0);
                    if (!__any_sync(0xffffffffu, act)) break;
                    step(y1);
                    if (!__any_sync(0xffffffffu, act)) break;
                    step(y2);
                    if (!__any_sync(0xffffffffu, act)) break;
                    step(y3);
                }
                if (gl == 0 && run < RA) ta[run] = t;
            }
        }
        __syncthreads();
        if (s_count > (uint32_t)MT_POOL) {                             // clustered keys: redo with tables
            if (threadIdx.x == 0) atomicExch(P.err, 1);
            return;
        }
        // ---- half b: keys in [lo - Wc, hi + Wc), each looked up in the table
        const uint64_t base = k ? lo - Wc : 0ull;
        const uint64_t span = (k == NB - 1) ? 0ull - base : lo + U + Wc - base;
        const uint64_t nxtb = k ? U : U - Wc;                             // next unit's base - base
        const uint64_t lob = lo - base;                                   // key - lo = (key - base) - lob
        for (int run = gid; run - gi < RB; run += NG) {
            bool act = run < RB;
            const int rr = act ? run : 0;
            const uint64_t xbb = xb[rr] - base;
            const uint32_t jj = j0b[rr];
            const uint32_t t0 = act ? tb[rr] : 0u;
            uint32_t t = t0;
            uint64_t y0 = Yb[(jj + t + gl) & lmb], y1 = Yb[(jj + t + GL + gl) & lmb];
            uint64_t y2 = Yb[(jj + t + 2 * GL + gl) & lmb], y3 = Yb[(jj + t + 3 * GL + gl) & lmb];
            auto step = [&](uint64_t& y) {
                const uint64_t rk = xbb + (y & ~(uint64_t)lmb);
                const bool in = act && t + gl < Nb && rk < span;
                const int pb = (int)((long long)(rk - lob) >> fsh);
                enqueue(in && maybe(pb), pb, (uint32_t)run, (uint32_t)y);
                const uint32_t cnt = __popc((__ballot_sync(0xffffffffu, in) >> gsh) & gbits);
                t += cnt;
                act = act && cnt == (uint32_t)GL;
                y = Yb[(jj + t + 3 * GL + gl) & lmb];
            };
            for (;;) {
                if (!__any_sync(0xffffffffu, act)) break;
                step(y0);
                if (!__any_sync(0xffffffffu, act)) break;
                step(y1);
                if (!__any_sync(0xffffffffu, act)) break;
                step(y2);
                if (!__any_sync(0xffffffffu, act)) break;
                step(y3);
            }
            // next unit's start: the first key >= its lo - Wc, i.e. with key - base >= nxtb;
            // those keys close the stretch [t0, t), so look back from its end
            if (gl == 0 && run < RB) {
                uint32_t nt = t;
                if (t > t0 && xbb + (Yb[(jj + t - 1) & lmb] & ~(uint64_t)lmb) >= nxtb) {
                    uint32_t lo_i = t0, hi_i = t - 1;                    // keys in the band: search
                    while (lo_i < hi_i) {
                        const uint32_t mid = (lo_i + hi_i) >> 1;
                        if (xbb + (Yb[(jj + mid) & lmb] & ~(uint64_t)lmb) < nxtb) lo_i = mid + 1; else hi_i = mid;
                    }
                    nt = lo_i;
                }
                tb[run] = nt;
            }
        }
        // circular wrap: unit 0 also meets keys of b in [2^64 - Wc, 2^64), the last unit keys in [0, Wc)
        if (k == 0)
            for (int g = warp; g < RB; g += nwarps) {
                const uint32_t s0 = run_lower_bound(Yb, j0b[g], Nb, xb[g], keepb, 0ull - Wc);
                walk_b(g, s0, 0ull - Wc, Wc, lo);
            }
        if (k == NB - 1)
            for (int g = warp; g < RB; g += nwarps) walk_b(g, 0u, 0ull, Wc, lo);
        drain();
        __syncthreads();
    }
}

// Exact re-check of the fingerprint hits of problem blockIdx.x / cpl: Tr_1 within
// W (Eq. 9 / Eq. 19, circular), then Tr_2 within W2, from the two pattern masks.
__global__ void __launch_bounds__(256) k_mitm_check(const MitmJob* __restrict__ js, int cpl) {
    __shared__ uint64_t wa[32], w2a[32], wb[32], w2b[32];
    const MitmJob& P = js[blockIdx.x / cpl];
    const int c = blockIdx.x % cpl;
    if (threadIdx.x < P.n_a) { wa[threadIdx.x] = P.w_a[threadIdx.x]; w2a[threadIdx.x] = P.w2_a[threadIdx.x]; }
    if (threadIdx.x < P.n_b) { wb[threadIdx.x] = P.w_b[threadIdx.x]; w2b[threadIdx.x] = P.w2_b[threadIdx.x]; }
    __syncthreads();
    unsigned long long nh = *P.nhits;
    if (nh > P.hcap) nh = P.hcap;
    unsigned long long n_pre = 0;
    for (unsigned long long i = (unsigned long long)c * blockDim.x + threadIdx.x; i < nh; i += (unsigned long long)cpl * blockDim.x) {
        const uint64_t h = P.hits[i];
        const uint32_t ma = (uint32_t)h, mb = (uint32_t)(h >> 32);
        const uint64_t v = mask_sum(wa, ma) + mask_sum(wb, mb);
        if (circ_dist(v) <= P.W) {
            ++n_pre;
            const uint64_t t2 = mask_sum(w2a, ma) + mask_sum(w2b, mb);
            if (circ_dist(t2) <= P.W2) {
                if (ma == 0 && mb == 0) {
                    P.ctr[3] = 1ull;
                } else {
                    const unsigned long long idx = atomicAdd(&P.ctr[2], 1ull);
                    if (idx < P.cap) P.cand[idx] = (uint64_t)ma | ((uint64_t)mb << P.n_a);
                }
            }
        }
    }
    if (n_pre) atomicAdd(&P.ctr[1], n_pre);
    if (c == 0 && threadIdx.x == 0) atomicAdd(&P.ctr[0], nh);
}

bool g_mitm_attr = false;

cudaError_t mitm_attrs() {
    if (g_mitm_attr) return cudaSuccess;
    cudaError_t e = cudaFuncSetAttribute(k_ybuild_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YS_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ymerge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YM_SMEM);
    if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mitm, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
    if (e == cudaSuccess) g_mitm_attr = true;
    return e;
}

// Launch the list build for the jobs d_yj[0..nh), sorted by l descending (host copy yj).
void build_lists(const YJob* yj, int nh, YJob* d_yj, cudaStream_t s) {
    k_ybuild_smem<<<nh, YS_THREADS, YS_SMEM, s>>>(d_yj);
    for (int i = YS_LOG; i < yj[0].l; ++i) {
        int nhi = 0;
        while (nhi < nh && yj[nhi].l > i) ++nhi;
        const int cpl = (2 << i) / YM_TILE;
        k_ysplit<<<(nhi * (cpl + 1) + 127) / 128, 128, 0, s>>>(d_yj, nhi, i, cpl);
        k_ymerge<<<nhi * cpl, YM_THREADS, YM_SMEM, s>>>(d_yj, i, cpl);
    }
}

}  // namespace

bool mitm_geometry(int n_a, int n_b, uint64_t W, MatchGeom* g) {
    if (n_a < 2 || n_b < n_a || n_b > 31) return false;
    auto lsplit = [](int h) { return h <= 10 ? h : (h - 7 < 10 ? 10 : (h - 7 > 21 ? 21 : h - 7)); };
    const int la = lsplit(n_a), lb = lsplit(n_b);
    if ((1 << (n_a - la)) > MT_RUNS || (1 << (n_b - lb)) > MT_RUNS) return false;
    int d1 = n_a - 13;
    if (d1 < 2) d1 = 2;
    const int su = 64 - d1;
    // keys in the lists carry the rounding of the low weights: <= l * 2^(l-1) per half
    const uint64_t wc = W + (uint64_t)la * (1ull << (la > 0 ? la - 1 : 0)) + (uint64_t)lb * (1ull << (lb > 0 ? lb - 1 : 0)) + 2;
    if (wc < W) return false;
    // a key's window must touch at most two bins: bin width 2^(su - nbl) > 2 Wc
    int nbl = MT_NBL;
    while (nbl >= 4 && !(wc < (1ull << (su - nbl - 1)))) --nbl;
    if (nbl < 4) return false;
    const int fsh = su - nbl - 16;
    const uint32_t NB = 1u << d1;
    uint32_t slab = NB / 256;
    if (slab < 1) slab = 1;
    if (slab > 64) slab = 64;
    memset(g, 0, sizeof(*g));
    g->fused = true;
    g->optimistic = true;
    g->n_a = n_a; g->n_b = n_b; g->d1 = d1; g->wc = wc;
    g->l_a = la; g->l_b = lb;
    g->nbl = nbl; g->slab = (int)slab;
    g->wf = (int)((wc >> fsh) + 1);
    g->bytes = match_bytes(*g);
    return true;
}

// Fingerprint hits of one problem: pairs with |K_a - K_b| below (wf + 1) 2^fsh,
// expected 2^(n_a + n_b) (2 wf + 3) 2^fsh / 2^64; room for 4x that + 2^16.
uint64_t mitm_hit_cap(const MatchGeom& g) {
    const int fsh = (64 - g.d1) - g.nbl - 16;
    const double e = std::ldexp((double)(2 * g.wf + 3), g.n_a + g.n_b + fsh - 64);
    const double all = std::ldexp(1.0, g.n_a + g.n_b);
    const double cap = std::min(all, 4.0 * e + 65536.0);
    return (uint64_t)cap + 1;
}

size_t mitm_half_bytes(int l) {
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    size_t b = a256((size_t)8 << l);
    if (l > YS_LOG) b += 2 * a256((size_t)8 << (l - 1)) + a256((((size_t)1 << l) / YM_TILE + 2) * 4);
    return b;
}

void mitm_layout_half(int l, char*& p, HalfJob* h) {
    auto take = [&](size_t bytes) { char* q = p; p += (bytes + 255) & ~(size_t)255; return q; };
    h->ylist = (uint64_t*)take((size_t)8 << l);
    h->ytmp = h->kb1 = nullptr;
    h->ysplit = nullptr;
    if (l > YS_LOG) {
        h->ytmp = (uint64_t*)take((size_t)8 << (l - 1));
        h->kb1 = (uint64_t*)take((size_t)8 << (l - 1));
        h->ysplit = (uint32_t*)take((((size_t)1 << l) / YM_TILE + 2) * 4);
    }
}

int mitm_launches(const ProbJob* const* F, int nF) {
    int maxl = 0;
    for (int i = 0; i < nF; ++i) maxl = std::max(maxl, std::max(F[i]->A.l, F[i]->B.l));
    return nF ? 3 + 2 * std::max(0, maxl - YS_LOG) : 0;
}

cudaError_t run_mitm(const ProbJob* const* F, int nF, void* dev_mjobs, void* dev_yjobs, cudaStream_t s,
                     cudaEvent_t ev_lists, cudaEvent_t ev_lists2) {
    static_assert(sizeof(MitmJob) <= sizeof(ProbJob), "MitmJob must fit a ProbJob slot");
    static_assert(sizeof(YJob) <= sizeof(HalfJob), "YJob must fit a HalfJob slot");
    if (nF <= 0) return cudaSuccess;
    cudaError_t e;
    e = mitm_attrs();
    if (e != cudaSuccess) return e;
    std::vector<YJob> yj;
    yj.reserve(2 * (size_t)nF);
    for (int i = 0; i < nF; ++i) {
        const HalfJob* hh[2] = {&F[i]->A, &F[i]->B};
        for (const HalfJob* h : hh) {
            YJob y;
            y.w = h->w; y.l = h->l; y.neg = h->neg;
            y.kb[0] = h->ytmp; y.kb[1] = h->kb1;
            y.splits = h->ysplit;
            y.ylist = h->ylist;
            yj.push_back(y);
        }
    }
    std::stable_sort(yj.begin(), yj.end(), [](const YJob& a, const YJob& b) { return a.l > b.l; });
    YJob* d_yj = (YJob*)dev_yjobs;
    e = cudaMemcpyAsync(d_yj, yj.data(), sizeof(YJob) * yj.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    build_lists(yj.data(), (int)yj.size(), d_yj, s);
    if (ev_lists) cudaEventRecord(ev_lists, s);
    if (ev_lists2) cudaEventRecord(ev_lists2, s);
    std::vector<MitmJob> mj(nF);
    int ctas = 0;
    for (int i = 0; i < nF; ++i) {
        const ProbJob& P = *F[i];
        MitmJob& m = mj[i];
        memset(&m, 0, sizeof(m));
        m.ya = P.A.ylist; m.yb = P.B.ylist;
        m.w_a = P.w_a; m.w2_a = P.w2_a; m.w_b = P.w_b; m.w2_b = P.w2_b;
        m.n_a = P.n_a; m.n_b = P.n_b; m.l_a = P.A.l; m.l_b = P.B.l;
        m.d1 = P.d1; m.nbl = P.nbl; m.slab = P.slab; m.wf = P.wf;
        m.cta_base = ctas;
        m.W = P.W; m.W2 = P.W2; m.Wc = P.Wc;
        m.cand = P.cand; m.cap = P.cap; m.ctr = P.ctr; m.err = P.A.err;
        m.hits = P.hits; m.nhits = P.ctr + 5; m.hcap = P.hcap;          // counters[5]: fingerprint hits
        // key-range shard: slabs [lo, hi) of this problem's (1 << d1) / slab
        const int slabs = (1 << P.d1) / P.slab;
        const int ns = P.nshards > 1 ? P.nshards : 1, sh = P.nshards > 1 ? P.shard : 0;
        const int lo = (int)((int64_t)slabs * sh / ns), hi = (int)((int64_t)slabs * (sh + 1) / ns);
        m.c_lo = lo;
        ctas += hi - lo;
    }
    MitmJob* d_mj = (MitmJob*)dev_mjobs;
    e = cudaMemcpyAsync(d_mj, mj.data(), sizeof(MitmJob) * nF, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    if (ctas > 0) k_mitm<<<ctas, MT_THREADS, MT_SMEM, s>>>(d_mj, nF);
    k_mitm_check<<<nF * 64, 256, 0, s>>>(d_mj, 64);
    return cudaGetLastError();
}

}  // namespace rfr

using namespace rfr;

// Stage entry: one half's sorted low-subset list (see include/rfr_stages.h).
extern "C" size_t rfr_stage_lowlist_workspace(int l) {
    if (l < 0 || l > 21) return 0;
    size_t b = 512;                                           // the job
    if (l > YS_LOG) b += 2 * (((size_t)8 << (l - 1)) + 256) + ((((size_t)1 << l) / YM_TILE + 2) * 4 + 256);
    return b;
}

extern "C" int rfr_stage_lowlist(const uint64_t* w, int l, int negate, uint64_t* list,
                                 void* workspace, size_t workspace_bytes, void* stream) {
    if (l < 0 || l > 21 || (l && !w) || !list || !workspace) return RFR_E_INVALID;
    if (((uintptr_t)workspace) & 255) return RFR_E_INVALID;
    if (workspace_bytes < rfr_stage_lowlist_workspace(l)) return RFR_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (mitm_attrs() != cudaSuccess) return RFR_E_CUDA;
    char* p = (char*)workspace;
    YJob* d_yj = (YJob*)p;
    p += 512;
    YJob y;
    memset(&y, 0, sizeof(y));
    y.w = w; y.l = l; y.neg = negate ? 1 : 0; y.ylist = list;
    if (l > YS_LOG) {
        y.kb[0] = (uint64_t*)p; p += ((size_t)8 << (l - 1)) + 256;
        y.kb[1] = (uint64_t*)p; p += ((size_t)8 << (l - 1)) + 256;
        y.splits = (uint32_t*)p;
    }
    if (cudaMemcpyAsync(d_yj, &y, sizeof(y), cudaMemcpyHostToDevice, s) != cudaSuccess) return RFR_E_CUDA;
    build_lists(&y, 1, d_yj, s);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
