// k_mitm.cu — fused meet-in-the-middle match (K-c + K-d + K-e of Section 3.3
// for large halves, with no key tables in device memory).
//
// Each half's h elements are split into low elements 0..l-1 and high
// elements l..h-1.  The sorted list Y of all 2^l exact low-subset sums (mod
// 2^64), with the subset mask of every entry in a parallel array, is built
// once per half by merging (k_ybuild_smem, k_ymerge: the sorted list of a set
// plus one element is the merge of the list and its copy shifted by the
// element's weight).  A directory D over the list's values (D[q] = the first
// entry >= q 2^(64-l)) finds the entry where any value would go in a couple of
// probes.  Every high subset x gives one run x + Y, so a half is 2^(h-l) <= 128
// runs, and the keys of a run inside any key range are one contiguous stretch
// of Y (circularly), found with two directory look-ups.
//
// The key space [0, 2^64) is cut into 2^d1 units of width U.  One CTA walks a
// slab of consecutive units; each warp owns up to four runs of each half.  Per
// unit
//   1. every warp appends the keys of its half-a runs that lie in the unit to
//      a shared-memory table (a 16-bit fingerprint of the key's position in
//      the unit, the run and list index, one linked list per bin) at slots
//      given by a prefix sum of the stretch lengths, and marks the cells the
//      key's window touches in an occupancy bitmap;
//   2. every warp reads the keys of its half-b runs within Wc of the unit,
//      [lo - Wc, hi + Wc) (circularly), tests one bitmap cell each and, for
//      the few keys whose cell is marked, walks the lists of the bins around
//      it (queued per warp and walked 32 at a time).
// A pair (a, b) with |K_a - K_b| <= Wc (keys of half b are negated sums, so
// K_a - K_b is the pattern's Tr_1 value) is met exactly once, in the unit
// holding K_a.  Fingerprint hits are re-checked exactly by k_mitm_check
// against the Tr_1 window W (Eq. 9 / Eq. 19, circular) and the Tr_2 window
// W2, so the candidate set is the same as RECOMBINE_C's.
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>
#include "k_match.cuh"
#include "rfr_device.cuh"
#include "rfr_stages.h"

namespace rfr {
namespace {

constexpr int YS_LOG = 13;                                     // list levels built in shared memory
constexpr int YS_THREADS = 1024;
constexpr size_t YS_SMEM = ((size_t)2 << YS_LOG) * (8 + 4);    // two (key, mask) buffers of 2^13 entries
constexpr int YM_THREADS = 128;
constexpr int YM_PER = 4;                                      // merge outputs per thread (512-output tiles)
constexpr int L_MAX = 25;                                      // list bits (2^7 runs of a 32-element half)

#ifndef RFR_MT_THREADS
#define RFR_MT_THREADS 1024
#endif
constexpr int MT_THREADS = RFR_MT_THREADS;
constexpr int MT_WARPS = MT_THREADS / 32;
constexpr int MT_UNIT_LOG = 14;                                // table-a keys of one unit: 2^14 on average
constexpr int MT_CAP = 24576;                                  // table slots (1.5 x the mean)
constexpr int MT_NBL = 13;                                     // at most 2^13 bins per unit (2 keys per bin)
constexpr int MT_HEADS = (1 << MT_NBL) + 4;                    // bins 0 .. 2^nbl (positions carry an offset)
constexpr int MT_RUNS = 128;                                   // at most 128 runs per half
constexpr int MT_RPW = MT_RUNS / MT_WARPS;                     // runs of each half per warp
constexpr int GL = 32 / MT_RPW;                                // lanes walking one run together
constexpr int MT_CH = 8;                                       // units whose stretches are found together
constexpr int MT_BM_LOG = 19;                                  // occupancy bitmap: about 2^19 cells per unit
constexpr int MT_BMW = (1 << (MT_BM_LOG - 5)) + 4;             // + margin cells (16-byte multiple)
constexpr int MT_QCAP = 64;                                    // deferred lookups per warp
constexpr uint32_t MT_NIL = 0xffffffffu;
constexpr int MT_APOS = MT_RPW * (MT_CH + 1);                  // per warp: half-a stretch starts
constexpr int MT_BPOS = MT_RPW * MT_CH * 2;                    // per warp: half-b stretch ends
constexpr size_t MT_SMEM = (size_t)MT_CAP * 4 + (size_t)MT_HEADS * 4 + (size_t)MT_BMW * 4 +
                           (size_t)MT_WARPS * MT_QCAP * 8 + (size_t)MT_WARPS * (MT_APOS + MT_BPOS) * 4 +
                           (size_t)MT_RUNS * 2 * 4 + (size_t)MT_WARPS * 4 + (size_t)MT_WARPS * MT_RPW * 2 * 8;

__device__ __forceinline__ uint32_t lower_bound_keys(const uint64_t* K, uint32_t n, uint64_t v) {
    uint32_t lo = 0, hi = n;
    while (lo < hi) {
        const uint32_t mid = (lo + hi) >> 1;
        if (K[mid] < v) lo = mid + 1; else hi = mid;
    }
    return lo;
}

// The weight added to every sum of a list when element i joins it.
__device__ __forceinline__ uint64_t list_step(const uint64_t* w, int neg, int i) {
    return neg ? 0ull - w[i] : w[i];
}

// Outputs d0 .. d1-1 of the merge of the sorted entries (K, M)[0..n) with the
// sorted sequence B[t] = K[(r + t) mod n] + c, mask M[(r + t) mod n] | bit (K
// shifted by c, rotated to its smallest element; equal entries take K first).
// n is a power of two.
template <class Out>
__device__ __forceinline__ void merge_range(const uint64_t* __restrict__ K, const uint32_t* __restrict__ M,
                                            uint32_t n, uint32_t r, uint64_t c, uint32_t bit,
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
        if (b >= n || (a < n && ka <= kb)) { out(d, ka, M[a]); ++a; }
        else { out(d, kb, M[(r + b) & nm] | bit); ++b; }
    }
}

struct YJob {
    const uint64_t* w;          // the half's weights (elements 0..l-1 used)
    int l, neg;                 // list bits; keys are negated sums for half b
    uint64_t* kb[2];            // [2^(l-1)] intermediate levels, ping-pong (l > YS_LOG only)
    uint32_t* mb[2];            // [2^(l-1)] their masks
    uint64_t* ylist;            // [2^l] result, ascending
    uint32_t* ymask;            // [2^l] result masks
    uint32_t* ydir;             // [2^l + 1] directory (null: not built)
    uint32_t* y32;              // [2^l] bits fsh .. fsh + 31 of each entry (with the directory)
    int fsh;
    uint32_t* splits;           // [2^l / YM_TILE + 2]: a level's tile starts on the merge path, then its rotation
};

// Levels 0 .. min(l, 13) - 1 of one half's list in shared memory.
__global__ void __launch_bounds__(YS_THREADS) k_ybuild_smem(const YJob* __restrict__ js) {
    extern __shared__ __align__(16) uint64_t ys_sm[];
    uint64_t* Kb[2] = {ys_sm, ys_sm + (1 << YS_LOG)};
    uint32_t* Mb[2] = {reinterpret_cast<uint32_t*>(ys_sm + (2 << YS_LOG)),
                       reinterpret_cast<uint32_t*>(ys_sm + (2 << YS_LOG)) + (1 << YS_LOG)};
    const YJob J = js[blockIdx.x];
    const int s = J.l < YS_LOG ? J.l : YS_LOG;
    if (threadIdx.x == 0) { Kb[0][0] = 0ull; Mb[0][0] = 0u; }
    __syncthreads();
    for (int i = 0; i < s; ++i) {
        const uint32_t n = 1u << i;
        const uint64_t c = list_step(J.w, J.neg, i);
        const uint64_t* K = Kb[i & 1];
        const uint32_t* M = Mb[i & 1];
        uint64_t* KO = Kb[(i + 1) & 1];
        uint32_t* MO = Mb[(i + 1) & 1];
        const uint32_t r = lower_bound_keys(K, n, 0ull - c);   // first entry that wraps when c is added
        const uint32_t tot = 2 * n, per = (tot + blockDim.x - 1) / blockDim.x;
        const uint32_t d0 = min(tot, threadIdx.x * per), d1 = min(tot, d0 + per);
        if (d0 < d1)
            merge_range(K, M, n, r, c, 1u << i, d0, d1, [&](uint32_t d, uint64_t k, uint32_t m) { KO[d] = k; MO[d] = m; });
        __syncthreads();
    }
    const uint64_t* K = Kb[s & 1];
    const uint32_t* M = Mb[s & 1];
    uint64_t* out = s == J.l ? J.ylist : J.kb[0];
    uint32_t* mout = s == J.l ? J.ymask : J.mb[0];
    for (uint32_t j = threadIdx.x; j < (1u << s); j += blockDim.x) { out[j] = K[j]; mout[j] = M[j]; }
}

// Level i >= 13 (2^i entries -> 2^(i+1)) for every half with l > i; cpl CTAs per
// half, each writing a tile of YM_TILE outputs.  The CTA finds where its tile
// starts and ends on the merge path (precomputed by k_ysplit), reads the two
// input stretches into shared memory with coalesced loads and merges them there,
// YM_PER consecutive outputs per thread kept in registers (the two merge heads
// too, so each output costs one key load) and written with 16-byte stores.  The
// last level writes the list itself, its 32-bit positions and its directory.
constexpr int YM_TILE = YM_THREADS * YM_PER;
constexpr size_t YM_SMEM = (size_t)YM_TILE * (8 + 4);

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
    const uint64_t cs = list_step(J.w, J.neg, i);
    const uint32_t r = lower_bound_keys(K, n, 0ull - cs);
    J.splits[c] = merge_split(K, n, r, cs, (uint32_t)c * YM_TILE);
    if (c == 0) J.splits[cpl + 1] = r;
}

__global__ void __launch_bounds__(YM_THREADS) k_ymerge(const YJob* __restrict__ js, int i, int cpl) {
    extern __shared__ __align__(16) uint64_t ym_sm[];
    uint64_t* tin = ym_sm;                        // [YM_TILE]: the stretch of K, then of the shifted copy
    uint32_t* min_ = reinterpret_cast<uint32_t*>(ym_sm + YM_TILE);   // [YM_TILE]: their masks
    const YJob& J = js[blockIdx.x / cpl];
    const int c = blockIdx.x % cpl;
    const uint32_t n = 1u << i, nm = n - 1;
    const int p = (i - YS_LOG) & 1;
    const uint64_t* __restrict__ K = J.kb[p];
    const uint32_t* __restrict__ M = J.mb[p];
    const uint64_t cs = list_step(J.w, J.neg, i);
    const uint32_t bit = 1u << i;
    const uint32_t r = J.splits[cpl + 1];
    const uint32_t o0 = (uint32_t)c * YM_TILE;
    const uint32_t a0 = J.splits[c], a1 = J.splits[c + 1], b0 = o0 - a0;
    const uint32_t na = a1 - a0;                  // nb = YM_TILE - na
    {
        // all of this thread's loads are in flight before the first store
        uint64_t kv[YM_PER];
        uint32_t mv[YM_PER];
#pragma unroll
        for (int q = 0; q < YM_PER; ++q) {
            const uint32_t j = threadIdx.x + (uint32_t)q * YM_THREADS;
            const uint32_t src = j < na ? a0 + j : ((r + b0 + (j - na)) & nm);
            kv[q] = K[src];
            mv[q] = M[src];
        }
#pragma unroll
        for (int q = 0; q < YM_PER; ++q) {
            const uint32_t j = threadIdx.x + (uint32_t)q * YM_THREADS;
            tin[j] = j < na ? kv[q] : kv[q] + cs;
            min_[j] = j < na ? mv[q] : (mv[q] | bit);
        }
    }
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
    const bool last = i == J.l - 1;
    uint64_t* KO = last ? J.ylist : J.kb[p ^ 1];
    uint32_t* MO = last ? J.ymask : J.mb[p ^ 1];
    uint64_t ka = ia < na ? A[ia] : 0ull, kb = ib < nb ? Bv[ib] : 0ull;
    if (!(last && J.ydir)) {
        // outputs dl .. dl + 7 straight from registers: 64 B of keys, 32 B of masks
        uint64_t kq[YM_PER];
        uint32_t mq[YM_PER];
#pragma unroll
        for (int q = 0; q < YM_PER; ++q) {
            const bool ta = ib >= nb || (ia < na && ka <= kb);
            kq[q] = ta ? ka : kb;
            mq[q] = ta ? min_[ia] : min_[na + ib];
            if (ta) { ++ia; ka = ia < na ? A[ia] : 0ull; } else { ++ib; kb = ib < nb ? Bv[ib] : 0ull; }
        }
        ulonglong2* k2 = reinterpret_cast<ulonglong2*>(KO + o0 + dl);
#pragma unroll
        for (int q = 0; q < YM_PER / 2; ++q) k2[q] = make_ulonglong2(kq[2 * q], kq[2 * q + 1]);
        uint4* m4 = reinterpret_cast<uint4*>(MO + o0 + dl);
#pragma unroll
        for (int q = 0; q < YM_PER / 4; ++q) m4[q] = make_uint4(mq[4 * q], mq[4 * q + 1], mq[4 * q + 2], mq[4 * q + 3]);
        return;
    }
    // the last level also writes the list's directory and positions (as k_ydir does):
    // D[q] = j for every q in (Y[j-1] >> (64-l), Y[j] >> (64-l)]
    const int sh = 64 - J.l;
    const uint32_t N = 2u * n;
    uint64_t pv;                                  // the output before this thread's first
    if (dl == 0) {                                // the tile's: the larger of the two inputs' last entries before it
        const uint64_t pa = a0 ? K[a0 - 1] : 0ull, pb = b0 ? K[(r + b0 - 1) & nm] + cs : 0ull;
        pv = !a0 ? pb : (!b0 ? pa : (pa > pb ? pa : pb));
    } else {
        const uint64_t xa = ia ? A[ia - 1] : 0ull, xb = ib ? Bv[ib - 1] : 0ull;
        pv = !ia ? xb : (!ib ? xa : (xa > xb ? xa : xb));
    }
    uint64_t kq[YM_PER];
    uint32_t mq[YM_PER];
#pragma unroll
    for (int q = 0; q < YM_PER; ++q) {
        const bool ta = ib >= nb || (ia < na && ka <= kb);
        kq[q] = ta ? ka : kb;
        mq[q] = ta ? min_[ia] : min_[na + ib];
        if (ta) { ++ia; ka = ia < na ? A[ia] : 0ull; } else { ++ib; kb = ib < nb ? Bv[ib] : 0ull; }
    }
    ulonglong2* k2 = reinterpret_cast<ulonglong2*>(KO + o0 + dl);
#pragma unroll
    for (int q = 0; q < YM_PER / 2; ++q) k2[q] = make_ulonglong2(kq[2 * q], kq[2 * q + 1]);
    uint4* m4 = reinterpret_cast<uint4*>(MO + o0 + dl);
    uint4* y4 = reinterpret_cast<uint4*>(J.y32 + o0 + dl);
#pragma unroll
    for (int q = 0; q < YM_PER / 4; ++q) {
        m4[q] = make_uint4(mq[4 * q], mq[4 * q + 1], mq[4 * q + 2], mq[4 * q + 3]);
        y4[q] = make_uint4((uint32_t)(kq[4 * q] >> J.fsh), (uint32_t)(kq[4 * q + 1] >> J.fsh),
                           (uint32_t)(kq[4 * q + 2] >> J.fsh), (uint32_t)(kq[4 * q + 3] >> J.fsh));
    }
#pragma unroll
    for (int q = 0; q < YM_PER; ++q) {
        const uint32_t d = o0 + dl + q;
        const uint64_t v = kq[q];
        const uint64_t qp = d ? ((q ? kq[q - 1] : pv) >> sh) + 1 : 0ull;
        for (uint64_t x = qp; x <= (v >> sh); ++x) J.ydir[x] = d;
        if (d == N - 1)
            for (uint64_t x = (v >> sh) + 1; x <= N; ++x) J.ydir[x] = N;
    }
}

// Directory of each finished list: D[q] = the first index j with Y[j] >= q 2^(64-l),
// q = 0 .. 2^l (D[2^l] = 2^l).  Thread j writes D[q] = j for every q in
// (Y[j-1] >> (64-l), Y[j] >> (64-l)], and y32[j] = bits fsh .. fsh + 31 of Y[j];
// grid: blockIdx.y = half.
__global__ void __launch_bounds__(256) k_ydir(const YJob* __restrict__ js) {
    const YJob& J = js[blockIdx.y];
    if (!J.ydir || J.l < 1 || J.l > YS_LOG) return;           // longer lists: the last merge level wrote it
    const uint32_t N = 1u << J.l;
    const int s = 64 - J.l;
    for (uint32_t j = blockIdx.x * blockDim.x + threadIdx.x; j <= N; j += gridDim.x * blockDim.x) {
        const uint64_t y = j < N ? J.ylist[j] : 0ull;
        const uint64_t qp = j ? (J.ylist[j - 1] >> s) + 1 : 0ull;       // first q not yet before j
        const uint64_t qc = j < N ? (y >> s) : (uint64_t)N;
        for (uint64_t q = qp; q <= qc; ++q) J.ydir[q] = j;
        if (j < N) J.y32[j] = (uint32_t)(y >> J.fsh);
    }
}

struct MitmJob {
    const uint64_t* ya;  const uint64_t* yb;                 // sorted low lists (exact sums)
    const uint32_t* ya32; const uint32_t* yb32;              // their bits fsh .. fsh + 31
    const uint32_t* ma_; const uint32_t* mb_;                // their masks
    const uint32_t* da;  const uint32_t* db;                 // their directories
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
    uint64_t* hits;                                           // fingerprint hits: (run_a, j_a) | (run_b, j_b) << 32
    unsigned long long* nhits;
    uint64_t hcap;
};

__device__ __forceinline__ uint64_t mask_sum(const uint64_t* w, uint32_t m) {
    uint64_t s = 0;
    for (; m; m &= m - 1) s += w[__ffs(m) - 1];
    return s;
}

// The table-a keys of the bins around position pb (a half-b key with pattern
// bits mb): those within wf are fingerprint hits.  A hit's table slot e gives
// the half-a run (the last run whose slots start at or before e) and the list
// index; k_mitm_check re-checks the pair exactly.  Not inlined: only the few
// half-b keys whose bitmap cell is marked come here, and keeping this code out
// of the key loops leaves their registers alone.
__device__ __noinline__ void mitm_walk(uint32_t pbu, uint32_t mb, const uint32_t* E, const uint32_t* head,
                                       const uint32_t* rsb, const uint32_t* rp0, int wf, int pmax, int la,
                                       const MitmJob* P) {
    const int pb = (int)pbu;
    const int plo = pb - wf < 0 ? 0 : pb - wf;
    const int phi = pb + wf > pmax ? pmax : pb + wf;
    const uint32_t lma = (1u << la) - 1u;
    for (int bin = plo >> 16; bin <= (phi >> 16); ++bin) {
        uint32_t e = head[bin];
        for (int steps = 0; e < (uint32_t)MT_CAP && steps < MT_CAP; ++steps) {   // lists end in NIL; bounded anyway
            const uint32_t en = E[e];
            const int d = ((bin << 16) | (int)(en & 0xffffu)) - pb;
            if (d >= -wf && d <= wf) {
                int lo_o = 0, hi_o = MT_RUNS - 1;
                while (lo_o < hi_o) {
                    const int mid = (lo_o + hi_o + 1) >> 1;
                    if (rsb[mid] <= e) lo_o = mid; else hi_o = mid - 1;
                }
                const uint32_t run = (uint32_t)(lo_o / MT_RPW + MT_WARPS * (lo_o % MT_RPW));
                const uint32_t ma = (run << la) | ((rp0[lo_o] + (e - rsb[lo_o])) & lma);
                const unsigned long long idx = atomicAdd(P->nhits, 1ull);
                if (idx < P->hcap) P->hits[idx] = (uint64_t)ma | ((uint64_t)mb << 32);
                else atomicExch(P->err, 1);                          // more hits than room: redo with tables
            }
            e = en >> 16;
        }
    }
}

// Stretches of one warp's runs in units k .. k + CH - 1 (lane by lane): half
// a's stretch of unit k + v starts at apos[i][v] (and ends where unit k + v + 1
// starts); half b's, within Wc of the unit, spans bpos[i][v][0 .. 1].  Not
// inlined: it runs once per CH units.
__device__ __noinline__ void mitm_stretches(uint32_t k, int su, uint64_t Wc, int qa, int qb,
                                            const uint64_t* Ya, const uint32_t* Da, int la,
                                            const uint64_t* Yb, const uint32_t* Db, int lb,
                                            const uint64_t* wxa, const uint64_t* wxb, uint32_t* wap, uint32_t* wbp) {
    // A lane's (up to) four look-ups run in lockstep, so that their dependent
    // L2 loads (two directory entries, then the bucket's entries) overlap
    // instead of queueing one look-up behind the other.
    constexpr int NS = (MT_APOS + MT_BPOS + 31) / 32;
    const int lane = threadIdx.x & 31;
    const uint64_t U = 1ull << su;
    uint64_t val[NS];
    uint32_t lo[NS], hi[NS];
    const uint64_t* Y[NS];
    uint32_t* out[NS];
#pragma unroll
    for (int m = 0; m < NS; ++m) {
        const int e = lane + 32 * m;
        out[m] = nullptr;
        Y[m] = Ya;
        val[m] = 0;
        lo[m] = hi[m] = 0;
        if (e < MT_APOS) {
            const int i = e / (MT_CH + 1), v = e % (MT_CH + 1);
            if (i < qa) {
                val[m] = ((uint64_t)(k + v) << su) - wxa[i];
                const uint32_t q = (uint32_t)(val[m] >> (64 - la));
                lo[m] = Da[q]; hi[m] = Da[q + 1];
                out[m] = wap + e;
            }
        } else if (e < MT_APOS + MT_BPOS) {
            const int e2 = e - MT_APOS, i = e2 / (2 * MT_CH), v = (e2 % (2 * MT_CH)) >> 1, side = e2 & 1;
            if (i < qb) {
                const uint64_t l0 = (uint64_t)(k + v) << su;
                val[m] = (side ? l0 + U + Wc : l0 - Wc) - wxb[i];
                const uint32_t q = (uint32_t)(val[m] >> (64 - lb));
                Y[m] = Yb;
                lo[m] = Db[q]; hi[m] = Db[q + 1];
                out[m] = wbp + e2;
            }
        }
    }
    // binary search of each bucket (lower bound of val): at most 32 halvings
    for (int step = 0; step < 32; ++step) {
        bool any = false;
#pragma unroll
        for (int m = 0; m < NS; ++m) {
            if (lo[m] < hi[m]) {
                const uint32_t mid = (lo[m] + hi[m]) >> 1;
                if (Y[m][mid] < val[m]) lo[m] = mid + 1; else hi[m] = mid;
                any = true;
            }
        }
        if (!any) break;
    }
#pragma unroll
    for (int m = 0; m < NS; ++m)
        if (out[m]) *out[m] = lo[m];
    __syncwarp();
}

// Key positions.  A key K of unit [lo, lo + U) (half b: within Wc of it) sits at
// position p = (K - lo + Off) >> fsh, Off = coff 2^fsh, so that every position
// and the window around it are >= 0.  For a run with offset x, K = x + y over
// its list values y, and p = y32 + (x - lo + Off) >> fsh - c, where y32 holds
// bits fsh.. of y and c in {0, 1} is the carry out of the low fsh bits, which
// is not computed: positions may be one low, and the window wf counts that.
// PV list positions read per lane with one load (8 or 16 bytes), so a run's
// keys go in blocks of GL * PV from the PV-aligned start of its stretch (list
// lengths are powers of two, so an aligned group never straddles the wrap).
template <int PV> struct PosVec;
template <> struct PosVec<2> {
    __device__ __forceinline__ static void load(const uint32_t* y, uint32_t i, uint32_t (&v)[2]) {
        const uint2 t = reinterpret_cast<const uint2*>(y)[i >> 1];
        v[0] = t.x; v[1] = t.y;
    }
};
template <> struct PosVec<4> {
    __device__ __forceinline__ static void load(const uint32_t* y, uint32_t i, uint32_t (&v)[4]) {
        const uint4 t = reinterpret_cast<const uint4*>(y)[i >> 2];
        v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
    }
};

// WRAP: some problem of the launch has fsh > 32, so positions are taken modulo
// 2^(64 - fsh) (halves of fewer than 17 elements); otherwise the 32-bit sums
// need no mask.
// PV: positions per lane and load (PosVec): 2 while the launch's lists stay in
// L2 (finer blocks, fewer idle lanes at the end of a stretch), 4 when they
// stream from DRAM (whole 128-byte lines per group of lanes).
template <bool WRAP, int PV>
__global__ void __launch_bounds__(MT_THREADS, 1) k_mitm(const MitmJob* __restrict__ js, int np) {
    extern __shared__ __align__(16) unsigned char mt_sm[];
    uint32_t* E = reinterpret_cast<uint32_t*>(mt_sm);                   // [CAP] fingerprint | next slot << 16
    uint32_t* head = E + MT_CAP;                                        // [bins + 4] first slot of each bin
    uint32_t* bm = head + MT_HEADS;                                     // [BMW] cells near a table-a key
    uint2* queue = reinterpret_cast<uint2*>(bm + MT_BMW);               // [warps][QCAP] deferred lookups
    uint32_t* apos = reinterpret_cast<uint32_t*>(queue + MT_WARPS * MT_QCAP);   // [warps][RPW][CH+1]
    uint32_t* bpos = apos + MT_WARPS * MT_APOS;                         // [warps][RPW][CH][2]
    uint32_t* rsb = bpos + MT_WARPS * MT_BPOS;                          // [warps * RPW] first slot of each run
    uint32_t* rp0 = rsb + MT_RUNS;                                      // [warps * RPW] its first list index
    uint32_t* s_tot = rp0 + MT_RUNS;                                    // [warps] table-a keys of the unit
    uint64_t* xs = reinterpret_cast<uint64_t*>(s_tot + MT_WARPS);       // [warps][2][RPW] run offsets
    __shared__ uint64_t wa[32], wb[32];

    int jl = 0, jh = np - 1;                                            // last job with cta_base <= blockIdx.x
    while (jl < jh) {
        const int mid = (jl + jh + 1) >> 1;
        if (js[mid].cta_base <= (int)blockIdx.x) jl = mid; else jh = mid - 1;
    }
    const MitmJob& P = js[jl];
    const int c = blockIdx.x - P.cta_base + P.c_lo;
    const int n_a = P.n_a, n_b = P.n_b, la = P.l_a, lb = P.l_b;
    const uint32_t Na = 1u << la, Nb = 1u << lb;
    const uint32_t lma = Na - 1u, lmb = Nb - 1u;
    const int RA = 1 << (n_a - la), RB = 1 << (n_b - lb);
    const int d1 = P.d1, su = 64 - d1, nbl = P.nbl, fsh = su - nbl - 16;
    const uint64_t U = 1ull << su;
    const uint64_t Wc = P.Wc;
    const int wf = P.wf;
    const int nbins = 1 << nbl;
    const uint32_t kmask = WRAP && fsh > 32 ? (1u << (64 - fsh)) - 1u : 0xffffffffu;   // positions modulo 2^(64 - fsh)
    // cells of 2^rsh positions, wider than a key's window of 2 wf + 1
    int rsh = nbl + 16 > MT_BM_LOG ? nbl + 16 - MT_BM_LOG : 0;
    while ((1 << rsh) <= 2 * wf + 1) ++rsh;
    const int coff = 1 << rsh;
    const uint64_t Off = (uint64_t)coff << fsh;
    const int nbmw = (((1 << (nbl + 16)) >> rsh) + 2 + 31) >> 5;
    const int pmax = ((nbins + 1) << 16) - 1;                           // positions of bins 0 .. nbins
    const uint64_t* __restrict__ Ya = P.ya;
    const uint64_t* __restrict__ Yb = P.yb;
    const uint32_t* __restrict__ Ya32 = P.ya32;
    const uint32_t* __restrict__ Yb32 = P.yb32;
    const uint32_t* __restrict__ Da = P.da;
    const uint32_t* __restrict__ Db = P.db;
    const uint32_t k0 = (uint32_t)c * (uint32_t)P.slab, k1 = k0 + (uint32_t)P.slab;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int g = lane / GL, gl = lane % GL;                            // run group of this lane
    // this warp's runs: run warp + MT_WARPS i for i < qa (half a), i < qb (half b)
    const int qa = RA > warp ? min(MT_RPW, (RA - warp + MT_WARPS - 1) / MT_WARPS) : 0;
    const int qb = RB > warp ? min(MT_RPW, (RB - warp + MT_WARPS - 1) / MT_WARPS) : 0;
    uint32_t* wap = apos + warp * MT_APOS;
    uint32_t* wbp = bpos + warp * MT_BPOS;
    uint64_t* wxa = xs + warp * (2 * MT_RPW);
    uint64_t* wxb = wxa + MT_RPW;
    uint2* wq = queue + warp * MT_QCAP;

    if (threadIdx.x < n_a) wa[threadIdx.x] = P.w_a[threadIdx.x];
    if (threadIdx.x < n_b) wb[threadIdx.x] = P.w_b[threadIdx.x];
    __syncthreads();
    if (lane < qa) {
        uint64_t x = 0;
        for (uint32_t t = (uint32_t)(warp + MT_WARPS * lane); t; t &= t - 1) x += wa[la + __ffs(t) - 1];
        wxa[lane] = x;
    } else if (lane >= MT_RPW && lane < MT_RPW + qb) {
        uint64_t x = 0;
        for (uint32_t t = (uint32_t)(warp + MT_WARPS * (lane - MT_RPW)); t; t &= t - 1) x -= wb[lb + __ffs(t) - 1];
        wxb[lane - MT_RPW] = x;
    }
    __syncwarp();

    // Warp-uniform: queue the lanes whose lookup may hit; scan 32 queued lookups at a time.
    uint32_t qn = 0;
    auto enqueue = [&](bool need, uint32_t pb, uint32_t mb) {
        const uint32_t qbal = __ballot_sync(0xffffffffu, need);
        if (!qbal) return;
        if (need) wq[qn + __popc(qbal & lt)] = make_uint2(pb, mb);
        qn += __popc(qbal);
        if (qn >= 32) {
            __syncwarp();
            const uint2 e = wq[lane];
            const uint2 e2 = lane + 32 < (int)qn ? wq[lane + 32] : make_uint2(0u, 0u);
            __syncwarp();
            if (lane + 32 < (int)qn) wq[lane] = e2;
            qn -= 32;
            mitm_walk(e.x, e.y, E, head, rsb, rp0, wf, pmax, la, &P);
        }
    };

    for (uint32_t k = k0; k < k1; ++k) {
        const uint32_t u = (k - k0) % MT_CH;
        const uint64_t lo = (uint64_t)k << su;
        if (u == 0) mitm_stretches(k, su, Wc, qa, qb, Ya, Da, la, Yb, Db, lb, wxa, wxb, wap, wbp);
        // reset the table heads and the bitmap with 16-byte stores
        {
            uint4* h4 = reinterpret_cast<uint4*>(head);
            for (int b = threadIdx.x; b < ((nbins + 4) >> 2); b += blockDim.x) h4[b] = make_uint4(MT_NIL, MT_NIL, MT_NIL, MT_NIL);
            uint4* b4 = reinterpret_cast<uint4*>(bm);
            for (int b = threadIdx.x; b < ((nbmw + 3) >> 2); b += blockDim.x) b4[b] = make_uint4(0u, 0u, 0u, 0u);
        }
        // this lane's half-a run (group g): stretch [p0, p0 + cnt) of the list, circularly
        uint32_t pa0 = 0, acnt = 0, apx = 0;
        if (g < qa) {
            pa0 = wap[g * (MT_CH + 1) + u];
            const uint32_t p1 = wap[g * (MT_CH + 1) + u + 1];
            const uint64_t v0 = lo - wxa[g];
            acnt = v0 >= 0ull - U ? Na - pa0 + p1 : p1 - pa0;              // the stretch wraps past the list's end
            apx = (uint32_t)((Off - v0) >> fsh);
        }
        uint32_t gpre = 0, wtot = 0;                                     // keys of the lower groups; of the warp
#pragma unroll
        for (int i = 0; i < MT_RPW; ++i) {
            const uint32_t ci = __shfl_sync(0xffffffffu, acnt, i * GL);
            gpre += i < g ? ci : 0u;
            wtot += ci;
        }
        // table a's first block of positions is loaded before the barrier, so the
        // load overlaps the barrier wait and the slot prefix sum
        constexpr uint32_t BS = GL * PV;                              // keys of a run per block
        const uint32_t a_al = pa0 & ~(uint32_t)(PV - 1), aoff = pa0 - a_al;
        uint32_t yn[PV];
        PosVec<PV>::load(Ya32, (a_al + PV * gl) & lma, yn);
        if (lane == 0) s_tot[warp] = wtot;
        __syncthreads();
        // slot base of this warp: table-a keys of the lower warps
        const uint32_t tv = lane < MT_WARPS ? s_tot[lane] : 0u;
        uint32_t incl = tv;
        for (int o = 1; o < 32; o <<= 1) {
            const uint32_t y = __shfl_up_sync(0xffffffffu, incl, o);
            if (lane >= o) incl += y;
        }
        const uint32_t T = __shfl_sync(0xffffffffu, incl, 31);
        const uint32_t sbg = __shfl_sync(0xffffffffu, incl - tv, warp) + gpre;
        if (T > (uint32_t)MT_CAP) {                                     // clustered keys: redo with tables
            if (threadIdx.x == 0) atomicExch(P.err, 1);
            return;
        }
        if (gl == 0) { rsb[warp * MT_RPW + g] = sbg; rp0[warp * MT_RPW + g] = pa0; }
        // ---- table a: every key of the unit, 8 lanes per run, 4 runs per warp
        {
            // blocks of BS list positions per run, PV per lane read with one load
            // from the aligned start a_al <= pa0; the next block's load is issued
            // before this block's keys are inserted
            const uint32_t itn = (__reduce_max_sync(0xffffffffu, acnt + aoff) + BS - 1) / BS;
            for (uint32_t it = 0; it < itn; ++it) {
                uint32_t y4[PV];
#pragma unroll
                for (int j = 0; j < PV; ++j) y4[j] = yn[j];
                if (it + 1 < itn) PosVec<PV>::load(Ya32, (a_al + (it + 1) * BS + PV * gl) & lma, yn);
#pragma unroll
                for (int j = 0; j < PV; ++j) {
                    const uint32_t t = it * BS + PV * gl + j - aoff;     // key index in the stretch
                    if (t < acnt) {
                        // a key of the unit sits at p in [coff - 1, 2^(nbl+16) + coff - 1]
                        // (coff = 2^rsh > 2 wf + 1, rsh <= 16), so p >> 16 <= nbins, p >= wf,
                        // and (p + wf) >> (rsh + 5) < MT_BMW: the indices need no clamp
                        const uint32_t p = (y4[j] + apx) & kmask;
                        const uint32_t slot = sbg + t;
                        const uint32_t old = atomicExch(&head[p >> 16], slot);
                        E[slot] = (p & 0xffffu) | (old << 16);
                        const uint32_t q0 = (p - (uint32_t)wf) >> rsh, q1 = (p + (uint32_t)wf) >> rsh;
                        atomicOr(&bm[q0 >> 5], (q1 != q0 ? 3u : 1u) << (q0 & 31));
                        if (q1 != q0 && (q0 & 31) == 31) atomicOr(&bm[q1 >> 5], 1u);
                    }
                }
            }
        }
        // ---- half b: keys in [lo - Wc, hi + Wc), each looked up in the table
        {
            uint32_t pb0 = 0, bcnt = 0, bpx = 0;
            if (g < qb) {
                pb0 = wbp[(g * MT_CH + u) * 2];
                const uint32_t p1 = wbp[(g * MT_CH + u) * 2 + 1];
                const uint64_t v0 = lo - Wc - wxb[g];
                bcnt = v0 + U + 2 * Wc < v0 ? Nb - pb0 + p1 : p1 - pb0;
                bpx = (uint32_t)((wxb[g] - lo + Off) >> fsh);
            }
            const uint32_t gbits = (uint32_t)(warp + MT_WARPS * g) << lb;
            // blocks of BS positions per run as in table a
            const uint32_t b_al = pb0 & ~(uint32_t)(PV - 1), boff = pb0 - b_al;
            const uint32_t itn = (__reduce_max_sync(0xffffffffu, bcnt + boff) + BS - 1) / BS;
            uint32_t yn[PV];
            PosVec<PV>::load(Yb32, (b_al + PV * gl) & lmb, yn);
            // the table and bitmap are complete past this barrier; half b's stretch
            // and first block were read before it, overlapping the wait
            __syncthreads();
            for (uint32_t it = 0; it < itn; ++it) {
                uint32_t y4[PV];
#pragma unroll
                for (int j = 0; j < PV; ++j) y4[j] = yn[j];
                if (it + 1 < itn) PosVec<PV>::load(Yb32, (b_al + (it + 1) * BS + PV * gl) & lmb, yn);
#pragma unroll
                for (int j = 0; j < PV; ++j) {
                    const uint32_t r = it * BS + PV * gl + j;            // index from b_al
                    const uint32_t p = (y4[j] + bpx) & kmask;
                    const uint32_t qc = p >> rsh;
                    const uint32_t wv = bm[min(qc >> 5, (uint32_t)(MT_BMW - 1))];
                    const bool need = r - boff < bcnt && ((wv >> (qc & 31)) & 1u);
                    enqueue(need, p, gbits | ((b_al + r) & lmb));
                }
            }
        }
        if (qn) {                                                          // the rest of the queue
            __syncwarp();
            if (lane < (int)qn) {
                const uint2 e = wq[lane];
                mitm_walk(e.x, e.y, E, head, rsb, rp0, wf, pmax, la, &P);
            }
            qn = 0;
        }
        __syncthreads();
    }
}

// Exact re-check of the fingerprint hits of problem blockIdx.x / cpl: Tr_1 within
// W (Eq. 9 / Eq. 19, circular), then Tr_2 within W2, from the two pattern masks
// (run bits above the low-list mask read at the hit's list index).
__global__ void __launch_bounds__(256) k_mitm_check(const MitmJob* __restrict__ js, int cpl) {
    __shared__ uint64_t wa[32], w2a[32], wb[32], w2b[32];
    const MitmJob& P = js[blockIdx.x / cpl];
    const int c = blockIdx.x % cpl;
    if (threadIdx.x < P.n_a) { wa[threadIdx.x] = P.w_a[threadIdx.x]; w2a[threadIdx.x] = P.w2_a[threadIdx.x]; }
    if (threadIdx.x < P.n_b) { wb[threadIdx.x] = P.w_b[threadIdx.x]; w2b[threadIdx.x] = P.w2_b[threadIdx.x]; }
    __syncthreads();
    const uint32_t lma = (1u << P.l_a) - 1u, lmb = (1u << P.l_b) - 1u;
    unsigned long long nh = *P.nhits;
    if (nh > P.hcap) nh = P.hcap;
    unsigned long long n_pre = 0;
    for (unsigned long long i = (unsigned long long)c * blockDim.x + threadIdx.x; i < nh; i += (unsigned long long)cpl * blockDim.x) {
        const uint64_t h = P.hits[i];
        const uint32_t ha = (uint32_t)h, hb = (uint32_t)(h >> 32);
        const uint32_t ma = (ha & ~lma) | P.ma_[ha & lma];
        const uint32_t mb = (hb & ~lmb) | P.mb_[hb & lmb];
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

PerDeviceOnce g_mitm_attr;

cudaError_t mitm_attrs() {
    return g_mitm_attr.run([] {
        cudaError_t e = cudaFuncSetAttribute(k_ybuild_smem, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YS_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_ymerge, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)YM_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mitm<false, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mitm<true, 2>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mitm<false, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
        if (e == cudaSuccess) e = cudaFuncSetAttribute(k_mitm<true, 4>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)MT_SMEM);
        return e;
    });
}

// Launch the list build for the jobs d_yj[0..nh), whose list bits, in launch
// order, are ls[0..nh) (descending), then the directories of the lists that
// have one and were finished in shared memory (the longest of those has
// dir_lmax bits; 0: none).
void build_lists(const int* ls, int nh, int dir_lmax, YJob* d_yj, cudaStream_t s) {
    k_ybuild_smem<<<nh, YS_THREADS, YS_SMEM, s>>>(d_yj);
    for (int i = YS_LOG; i < ls[0]; ++i) {
        int nhi = 0;
        while (nhi < nh && ls[nhi] > i) ++nhi;
        const int cpl = (2 << i) / YM_TILE;
        k_ysplit<<<(nhi * (cpl + 1) + 127) / 128, 128, 0, s>>>(d_yj, nhi, i, cpl);
        k_ymerge<<<nhi * cpl, YM_THREADS, YM_SMEM, s>>>(d_yj, i, cpl);
    }
    if (dir_lmax > 0) {
        const int bx = (int)std::min<uint64_t>(((1ull << dir_lmax) + 1 + 255) / 256, 4096);
        k_ydir<<<dim3(bx, nh), 256, 0, s>>>(d_yj);
    }
}

int lsplit(int h) { return h <= 10 ? h : std::max(10, h - 7); }

}  // namespace

bool mitm_geometry(int n_a, int n_b, uint64_t W, MatchGeom* g, const TuneParams* tp) {
    if (n_a < 2 || n_b < n_a || n_b > 32) return false;
    const int la = lsplit(n_a), lb = lsplit(n_b);
    if (la > L_MAX || lb > L_MAX || (1 << (n_a - la)) > MT_RUNS || (1 << (n_b - lb)) > MT_RUNS) return false;
    // units of 2^ulog half-a keys on average (the table holds 1.5 x 2^14), at most 2^nbl_max bins
    const int ulog = tp ? std::min(MT_UNIT_LOG, std::max(12, tp->unit_log)) : MT_UNIT_LOG;
    const int nbl_max = tp ? std::min(MT_NBL, std::max(10, tp->nbl_max)) : MT_NBL;
    int d1 = n_a - ulog;
    if (d1 < 2) d1 = 2;
    const int su = 64 - d1;
    // the lists hold exact sums: the coarse window only rounds up
    const uint64_t wc = W + 2;
    if (wc < W) return false;
    // a key's window (positions of 2^fsh, two more for the dropped carries) must
    // stay below half a bin of 2^16 positions: bin width 2^(su - nbl) > 4 Wc
    int nbl = nbl_max;
    while (nbl >= 4 && !(wc < (1ull << (su - nbl - 2)))) --nbl;
    if (nbl < 4) return false;
    const int fsh = su - nbl - 16;
    // k_mitm indexes its table heads and bitmap words from a half-a key's position
    // p in [coff - 1, 2^(nbl+16) + coff - 1] without clamps: check those bounds
    // for this geometry (cells of 2^rsh positions, as the kernel derives them)
    {
        const uint64_t wfh = (wc >> fsh) + 2;
        int rsh = nbl + 16 > MT_BM_LOG ? nbl + 16 - MT_BM_LOG : 0;
        while ((1ull << rsh) <= 2 * wfh + 1) ++rsh;
        const uint64_t coff = 1ull << rsh, pmax = (1ull << (nbl + 16)) + coff - 1;
        if ((pmax >> 16) > (1ull << nbl) || coff - 1 < wfh || ((pmax + wfh) >> rsh >> 5) >= (uint64_t)MT_BMW)
            return false;
    }
    const uint32_t NB = 1u << d1;
    // the slab length of a lone problem (run_mitm chooses it per launch): up to
    // MT_CH units, the stretch-search period, and at least 128 CTAs
    uint32_t slab = NB / 128;
    if (slab < 1) slab = 1;
    if (slab > (uint32_t)MT_CH) slab = MT_CH;
    memset(g, 0, sizeof(*g));
    g->fused = true;
    g->optimistic = true;
    g->n_a = n_a; g->n_b = n_b; g->d1 = d1; g->wc = wc;
    g->l_a = la; g->l_b = lb;
    g->nbl = nbl; g->slab = (int)slab;
    g->wf = (int)((wc >> fsh) + 2);
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

static size_t a256(size_t x) { return (x + 255) & ~(size_t)255; }

size_t mitm_half_bytes(int l) {
    size_t b = a256((size_t)8 << l) + 2 * a256((size_t)4 << l) + a256((((size_t)1 << l) + 1) * 4);
    if (l > YS_LOG) b += 2 * a256((size_t)8 << (l - 1)) + 2 * a256((size_t)4 << (l - 1)) +
                         a256((((size_t)1 << l) / YM_TILE + 2) * 4);
    return b;
}

void mitm_layout_half(int l, char*& p, HalfJob* h) {
    auto take = [&](size_t bytes) { char* q = p; p += a256(bytes); return q; };
    h->ylist = (uint64_t*)take((size_t)8 << l);
    h->ymask = (uint32_t*)take((size_t)4 << l);
    h->ydir = (uint32_t*)take((((size_t)1 << l) + 1) * 4);
    h->y32 = (uint32_t*)take((size_t)4 << l);
    h->ytmp = h->kb1 = nullptr;
    h->ymtmp[0] = h->ymtmp[1] = nullptr;
    h->ysplit = nullptr;
    if (l > YS_LOG) {
        h->ytmp = (uint64_t*)take((size_t)8 << (l - 1));
        h->kb1 = (uint64_t*)take((size_t)8 << (l - 1));
        h->ymtmp[0] = (uint32_t*)take((size_t)4 << (l - 1));
        h->ymtmp[1] = (uint32_t*)take((size_t)4 << (l - 1));
        h->ysplit = (uint32_t*)take((((size_t)1 << l) / YM_TILE + 2) * 4);
    }
}

int mitm_launches(const ProbJob* const* F, int nF) {
    // k_ybuild_smem, two per merge level, k_ydir when a list ends in shared
    // memory, k_mitm (when it has CTAs, which every fused problem gives) and k_mitm_check
    int maxl = 0;
    bool dir = false;
    for (int i = 0; i < nF; ++i) {
        maxl = std::max(maxl, std::max(F[i]->A.l, F[i]->B.l));
        dir = dir || (F[i]->A.ydir && F[i]->A.l <= YS_LOG) || (F[i]->B.ydir && F[i]->B.l <= YS_LOG);
    }
    return nF ? 3 + 2 * std::max(0, maxl - YS_LOG) + (dir ? 1 : 0) : 0;
}

cudaError_t mitm_prepare(const ProbJob* const* F, int nF, void* mj_host, void* yj_host, MitmShape* sh) {
    static_assert(sizeof(MitmJob) <= sizeof(ProbJob), "MitmJob must fit a ProbJob slot");
    static_assert(sizeof(YJob) <= sizeof(HalfJob), "YJob must fit a HalfJob slot");
    sh->nF = nF;
    sh->nh = 2 * nF;
    sh->ctas = 0;
    sh->dir_lmax = 0;
    sh->wrap = 0;
    sh->wide = 0;
    sh->ls.clear();
    if (nF <= 0) return cudaSuccess;
    const cudaError_t e = mitm_attrs();
    if (e != cudaSuccess) return e;
    std::vector<YJob> yj;
    yj.reserve(2 * (size_t)nF);
    for (int i = 0; i < nF; ++i) {
        const HalfJob* hh[2] = {&F[i]->A, &F[i]->B};
        for (const HalfJob* h : hh) {
            YJob y;
            y.w = h->w; y.l = h->l; y.neg = h->neg;
            y.kb[0] = h->ytmp; y.kb[1] = h->kb1;
            y.mb[0] = h->ymtmp[0]; y.mb[1] = h->ymtmp[1];
            y.splits = h->ysplit;
            y.ylist = h->ylist; y.ymask = h->ymask; y.ydir = h->ydir;
            y.y32 = h->y32; y.fsh = (64 - F[i]->d1) - F[i]->nbl - 16;
            yj.push_back(y);
        }
    }
    std::stable_sort(yj.begin(), yj.end(), [](const YJob& a, const YJob& b) { return a.l > b.l; });
    for (const YJob& y : yj) {
        sh->ls.push_back(y.l);
        if (y.ydir && y.l <= YS_LOG) sh->dir_lmax = std::max(sh->dir_lmax, std::max(1, y.l));
    }
    memcpy(yj_host, yj.data(), sizeof(YJob) * yj.size());
    // CTAs of the costliest units first (keys per unit of both halves), so that
    // the last wave holds the cheapest ones
    std::vector<int> order(nF);
    for (int i = 0; i < nF; ++i) order[i] = i;
    auto unit_cost = [&](int i) {
        return std::ldexp(1.0, F[i]->n_a - F[i]->d1) + std::ldexp(1.0, F[i]->n_b - F[i]->d1);
    };
    std::stable_sort(order.begin(), order.end(), [&](int x, int y) { return unit_cost(x) > unit_cost(y); });
    // slab length for this launch: the longest of 64, 32, 16, 8 units that still
    // gives 20 waves of CTAs (one per SM), so that the last wave is a small share;
    // a problem keeps at least 128 CTAs and at most its geometry's slab
    double tot_units = 0;
    for (int i = 0; i < nF; ++i) tot_units += std::ldexp(1.0, F[i]->d1);
    int sg = 64;
    while (sg > MT_CH && tot_units / sg < 20.0 * 148.0) sg /= 2;
    MitmJob* mj = (MitmJob*)mj_host;
    int ctas = 0;
    for (int oi = 0; oi < nF; ++oi) {
        const ProbJob& P = *F[order[oi]];
        MitmJob m;
        int slab = (1 << P.d1) / 128;
        if (slab > sg) slab = sg;
        if (slab < 1) slab = 1;
        memset(&m, 0, sizeof(m));
        m.ya = P.A.ylist; m.yb = P.B.ylist;
        m.ya32 = P.A.y32; m.yb32 = P.B.y32;
        m.ma_ = P.A.ymask; m.mb_ = P.B.ymask;
        m.da = P.A.ydir; m.db = P.B.ydir;
        m.w_a = P.w_a; m.w2_a = P.w2_a; m.w_b = P.w_b; m.w2_b = P.w2_b;
        m.n_a = P.n_a; m.n_b = P.n_b; m.l_a = P.A.l; m.l_b = P.B.l;
        m.d1 = P.d1; m.nbl = P.nbl; m.slab = slab; m.wf = P.wf;
        if ((64 - P.d1) - P.nbl - 16 > 32) sh->wrap = 1;
        // position lists of more than 32 MB per problem stream from DRAM: 16-byte loads
        if ((((size_t)1 << P.A.l) + ((size_t)1 << P.B.l)) * 4 > ((size_t)32 << 20)) sh->wide = 1;
        m.cta_base = ctas;
        m.W = P.W; m.W2 = P.W2; m.Wc = P.Wc;
        m.cand = P.cand; m.cap = P.cap; m.ctr = P.ctr; m.err = P.A.err;
        m.hits = P.hits; m.nhits = P.ctr + 5; m.hcap = P.hcap;          // counters[5]: fingerprint hits
        // key-range shard: slabs [lo, hi) of this problem's (1 << d1) / slab,
        // rounded up so that shard 0 always holds slab 0 (the trivial pair)
        const int slabs = (1 << P.d1) / slab;
        const int ns = P.nshards > 1 ? P.nshards : 1, shx = P.nshards > 1 ? P.shard : 0;
        const int lo = (int)(((int64_t)slabs * shx + ns - 1) / ns), hi = (int)(((int64_t)slabs * (shx + 1) + ns - 1) / ns);
        m.c_lo = lo;
        ctas += hi - lo;
        memcpy(&mj[oi], &m, sizeof(m));
    }
    sh->ctas = ctas;
    return cudaSuccess;
}

cudaError_t mitm_issue(const MitmShape& sh, void* dev_mjobs, void* dev_yjobs, cudaStream_t s,
                       cudaEvent_t ev_lists, cudaEvent_t ev_lists2, unsigned ev_flags) {
    if (sh.nF <= 0) return cudaSuccess;
    build_lists(sh.ls.data(), sh.nh, sh.dir_lmax, (YJob*)dev_yjobs, s);
    if (ev_lists) cudaEventRecordWithFlags(ev_lists, s, ev_flags);
    if (ev_lists2) cudaEventRecordWithFlags(ev_lists2, s, ev_flags);
    const MitmJob* d_mj = (const MitmJob*)dev_mjobs;
    if (sh.ctas > 0) {
        if (sh.wide) {
            if (sh.wrap) k_mitm<true, 4><<<sh.ctas, MT_THREADS, MT_SMEM, s>>>(d_mj, sh.nF);
            else k_mitm<false, 4><<<sh.ctas, MT_THREADS, MT_SMEM, s>>>(d_mj, sh.nF);
        } else {
            if (sh.wrap) k_mitm<true, 2><<<sh.ctas, MT_THREADS, MT_SMEM, s>>>(d_mj, sh.nF);
            else k_mitm<false, 2><<<sh.ctas, MT_THREADS, MT_SMEM, s>>>(d_mj, sh.nF);
        }
    }
    k_mitm_check<<<sh.nF * 64, 256, 0, s>>>(d_mj, 64);
    return cudaGetLastError();
}

size_t mitm_job_bytes(int nF) { return (size_t)nF * sizeof(MitmJob); }
size_t mitm_yjob_bytes(int nF) { return (size_t)2 * nF * sizeof(YJob); }

cudaError_t run_mitm(const ProbJob* const* F, int nF, void* dev_mjobs, void* dev_yjobs, cudaStream_t s,
                     cudaEvent_t ev_lists, cudaEvent_t ev_lists2) {
    if (nF <= 0) return cudaSuccess;
    std::vector<MitmJob> mj(nF);
    std::vector<YJob> yj(2 * (size_t)nF);
    MitmShape sh;
    cudaError_t e = mitm_prepare(F, nF, mj.data(), yj.data(), &sh);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dev_yjobs, yj.data(), sizeof(YJob) * yj.size(), cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dev_mjobs, mj.data(), sizeof(MitmJob) * nF, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return mitm_issue(sh, dev_mjobs, dev_yjobs, s, ev_lists, ev_lists2, cudaEventRecordDefault);
}

}  // namespace rfr

using namespace rfr;

// Stage entry: one half's sorted low-subset list (see include/rfr_stages.h).
extern "C" size_t rfr_stage_lowlist_workspace(int l) {
    if (l < 0 || l > L_MAX) return 0;
    size_t b = 512;                                           // the job
    if (l > YS_LOG) b += 2 * (((size_t)8 << (l - 1)) + 256) + 2 * (((size_t)4 << (l - 1)) + 256) +
                         ((((size_t)1 << l) / YM_TILE + 2) * 4 + 256);
    return b;
}

extern "C" int rfr_stage_lowlist(const uint64_t* w, int l, int negate, uint64_t* list, uint32_t* masks,
                                 void* workspace, size_t workspace_bytes, void* stream) {
    if (l < 0 || l > L_MAX || (l && !w) || !list || !masks || !workspace) return RFR_E_INVALID;
    if (((uintptr_t)workspace) & 255) return RFR_E_INVALID;
    if (workspace_bytes < rfr_stage_lowlist_workspace(l)) return RFR_E_INVALID;
    cudaStream_t s = (cudaStream_t)stream;
    if (mitm_attrs() != cudaSuccess) return RFR_E_CUDA;
    char* p = (char*)workspace;
    YJob* d_yj = (YJob*)p;
    p += 512;
    YJob y;
    memset(&y, 0, sizeof(y));
    y.w = w; y.l = l; y.neg = negate ? 1 : 0; y.ylist = list; y.ymask = masks;
    if (l > YS_LOG) {
        y.kb[0] = (uint64_t*)p; p += ((size_t)8 << (l - 1)) + 256;
        y.kb[1] = (uint64_t*)p; p += ((size_t)8 << (l - 1)) + 256;
        y.mb[0] = (uint32_t*)p; p += ((size_t)4 << (l - 1)) + 256;
        y.mb[1] = (uint32_t*)p; p += ((size_t)4 << (l - 1)) + 256;
        y.splits = (uint32_t*)p;
    }
    if (cudaMemcpyAsync(d_yj, &y, sizeof(y), cudaMemcpyHostToDevice, s) != cudaSuccess) return RFR_E_CUDA;
    build_lists(&y.l, 1, 0, d_yj, s);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
