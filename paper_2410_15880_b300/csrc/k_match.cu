// k_match.cu — K-c enumerate, K-d radix partition/sort, K-e match.
//
// Section 3.3 (RECOMBINE_C): split the searched elements into halves a and
// b, form every half-subset sum (EXPAND), sort, and find every pair whose
// sum is within the integrality window (FIND).  With keys
//     alpha(s_a) = sum_{i in s_a} w_a[i]          (mod 2^64)
//     beta'(s_b) = -sum_{i in s_b} w_b[i]         (mod 2^64)
// a pair is accepted iff |alpha - beta'| <= W on the circle, i.e. Eq. 9/19
// with the circular reading (sums near 0 and near 2^64 both count).
//
// Layout and passes (per problem, all problems of a batch in each launch):
//  * Radix digit 1 (top d1 key bits, 4..8192 buckets), produced from sorted
//    runs.  A half's h elements split into low bits 0..l-1 (l <= 16) and high
//    bits l..h-1:
//      k_ysort — list Y of the 2^l low-subset sums (low l key bits replaced by
//                the low mask), sorted by a stable LSD radix sort (one CTA);
//      k_runs<count>   — walks every run x + Y (one per high subset x);
//                the keys of a run rise, so the 32 lanes of a step fall into
//                a few buckets and one atomic per bucket group updates the
//                per-CTA histogram;
//      k_colscan / k_bscan — per-CTA offsets and bucket starts;
//      k_runs<scatter> — the same walk, each bucket group reserving
//                consecutive slots at the bucket's cursor and writing them.
//    Record (8 bytes): ((key << d1) & ~(2^h - 1)) | mask, key = x + (y with
//    its low l bits cleared).  The top d1 key bits are implied by the bucket;
//    the coarse key is below the true sum by less than 2^l + 2^max(0, h-d1).
//  * Radix digit 2 + K-e (k_join), one CTA per bucket: the bucket's table-a
//    records are counting-sorted by the next 13 key bits into shared memory
//    (chunks of 9216), then every table-b record of the bucket streams past
//    and probes the sub-buckets its coarse window covers.  Coarse hits are
//    re-checked exactly from the masks (full 64-bit sums of w), then the Tr_2
//    window filters them, then the pattern is appended to the candidate list.
//    Records of b whose window reaches a neighbouring bucket are also copied
//    into that bucket's halo list, so each (a, b) pair is examined by exactly
//    one CTA: the one owning a's bucket.
#include "rfr_device.cuh"
#include "k_match.cuh"
#include <cstring>
#include <vector>

namespace rfr {

template <class KeyF>
__device__ __forceinline__ int find_last_le(int n, int x, KeyF key) {
    int lo = 0, hi = n - 1;
    while (lo < hi) {
        int mid = (lo + hi + 1) >> 1;
        if (key(mid) <= x) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__device__ __forceinline__ uint64_t lowmask(int h) { return h ? (~0ull >> (64 - h)) : 0ull; }

// Visit every mask m in [m0, m0 + per) with key = sum_{i in m} sw[i] mod 2^64.
// per is a power of two; each thread walks chunks of up to 16 consecutive
// masks in Gray-code order (one add or subtract per step).
template <class F>
__device__ __forceinline__ void enumerate_range(const uint64_t* sw, uint64_t m0, uint64_t per, F&& f) {
    const int lg = per >= 16 ? 4 : (63 - __clzll((long long)per));
    const uint32_t E = 1u << lg;
    const uint64_t chunks = per >> lg;
    for (uint64_t q = threadIdx.x; q < chunks; q += blockDim.x) {
        const uint64_t ms = m0 + (q << lg);
        uint64_t key = 0;
        for (uint64_t t = ms; t; t &= t - 1) key += sw[__ffsll((long long)t) - 1];
        f(ms, key);
        for (uint32_t k = 1; k < E; ++k) {
            const int b = __ffs(k) - 1;
            const uint32_t g = k ^ (k >> 1);
            if ((g >> b) & 1u) key += sw[b]; else key -= sw[b];
            f(ms | g, key);
        }
    }
}

__device__ uint32_t block_excl_scan(uint32_t v, uint32_t* total, uint32_t* warp_sums) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nw = blockDim.x >> 5;
    uint32_t x = v;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        uint32_t y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
    }
    if (lane == 31) warp_sums[wid] = x;
    __syncthreads();
    if (wid == 0) {
        uint32_t s = lane < nw ? warp_sums[lane] : 0u;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            uint32_t y = __shfl_up_sync(0xffffffffu, s, o);
            if (lane >= o) s += y;
        }
        warp_sums[lane] = s;
    }
    __syncthreads();
    uint32_t ex = x - v + (wid ? warp_sums[wid - 1] : 0u);
    *total = warp_sums[nw - 1];
    __syncthreads();
    return ex;
}

// In-place exclusive scan of a[0..n), a[n] = total if write_total.  Two
// reads of a (the second after the block-wide scan of the per-thread sums).
__device__ void block_scan_array(uint32_t* a, int n, bool write_total, uint32_t* warp_sums) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < n) s += a[b0 + i];
    uint32_t total;
    uint32_t ex = block_excl_scan(s, &total, warp_sums);
    for (int i = 0; i < per; ++i) {
        if (b0 + i < n) {
            const uint32_t v = a[b0 + i];
            a[b0 + i] = ex;
            ex += v;
        }
    }
    if (write_total && threadIdx.x == 0) a[n] = total;
}

// Shared-memory arrays scanned with one contiguous chunk per thread are
// padded by one word every 32 (index s -> s + s/32): thread t's chunk then
// starts in bank (17 t) mod 32 and a warp's accesses never collide.
__host__ __device__ __forceinline__ int pad32(int s) { return s + (s >> 5); }

// In-place exclusive scan of a padded shared array a[pad32(0 .. n)).
__device__ void block_scan_padded(uint32_t* a, int n, uint32_t* warp_sums) {
    const int per = (n + blockDim.x - 1) / blockDim.x;
    const int b0 = threadIdx.x * per;
    uint32_t s = 0;
    for (int i = 0; i < per; ++i)
        if (b0 + i < n) s += a[pad32(b0 + i)];
    uint32_t total;
    uint32_t ex = block_excl_scan(s, &total, warp_sums);
    for (int i = 0; i < per; ++i) {
        if (b0 + i < n) {
            const uint32_t v = a[pad32(b0 + i)];
            a[pad32(b0 + i)] = ex;
            ex += v;
        }
    }
}

// ---------------------------------------------------------------- K-c plain
// keys[s] for s < 2^h in pattern order.  Lanes own mask bits 0..5 (bit 0 is
// the pair inside one 128-bit store), warps walk bits >= 6 in Gray order, so
// each warp step writes 64 consecutive keys (512 bytes).
__global__ void __launch_bounds__(256) k_enum_plain(const uint64_t* __restrict__ w, int h,
                                                    uint64_t* __restrict__ keys) {
    __shared__ uint64_t sw[32];
    if (threadIdx.x < h) sw[threadIdx.x] = w[threadIdx.x];
    __syncthreads();
    if (h < 6) {
        const uint32_t s = blockIdx.x * blockDim.x + threadIdx.x;
        if (s < (1u << h)) {
            uint64_t k = 0;
            for (int i = 0; i < h; ++i) if ((s >> i) & 1u) k += sw[i];
            keys[s] = k;
        }
        return;
    }
    const int lane = threadIdx.x & 31;
    const uint64_t gw = (blockIdx.x * (uint64_t)blockDim.x + threadIdx.x) >> 5;
    const uint64_t tw = ((uint64_t)gridDim.x * blockDim.x) >> 5;
    const uint64_t nhigh = 1ull << (h - 6);
    const uint64_t G = (nhigh + tw - 1) / tw;
    const uint64_t j0 = gw * G, j1 = min(nhigh, j0 + G);
    if (j0 >= j1) return;
    uint64_t lb = 0;
    for (int i = 1; i < 6; ++i) if ((lane >> (i - 1)) & 1) lb += sw[i];
    const uint64_t w0 = sw[0];
    uint64_t g = j0 ^ (j0 >> 1);
    uint64_t hk = 0;
    for (uint64_t t = g; t; t &= t - 1) hk += sw[6 + __ffsll((long long)t) - 1];
    for (uint64_t j = j0;;) {
        const uint64_t k0 = hk + lb;
        ulonglong2 v;
        v.x = k0;
        v.y = k0 + w0;
        reinterpret_cast<ulonglong2*>(keys + (g << 6))[lane] = v;
        if (++j >= j1) break;
        const int b = __ffsll((long long)j) - 1;
        const uint64_t gn = j ^ (j >> 1);
        if ((gn >> b) & 1ull) hk += sw[6 + b]; else hk -= sw[6 + b];
        g = gn;
    }
}

// ---------------------------------------------------------------- K-d: sorted low list
// One stable LSD pass over src[0..N) -> dst by the 8-bit digit at `shift`.
// Warp w owns the contiguous input chunk w; ranks inside a warp come from
// __match_any_sync, so equal digits keep their input order (stable).
__device__ void lsd_pass(const uint64_t* src, uint64_t* dst, uint32_t N, int shift,
                         uint32_t (*whist)[256], uint32_t* dbase, uint32_t* warp_sums) {
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const uint32_t chunk = (N + 31) / 32;
    const uint32_t b0 = min(N, (uint32_t)w * chunk), b1 = min(N, b0 + chunk);
    for (int d = lane; d < 256; d += 32) whist[w][d] = 0u;
    __syncwarp();
    for (uint32_t base = b0; base < b1; base += 32) {
        const uint32_t i = base + lane;
        const bool valid = i < b1;
        const uint64_t v = valid ? src[i] : 0ull;
        const uint32_t d = valid ? (uint32_t)((v >> shift) & 255u) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        if (valid && lane == __ffs(peers) - 1) whist[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
    uint32_t tot = 0;
    if (threadIdx.x < 256)
        for (int ww = 0; ww < 32; ++ww) {
            const uint32_t c = whist[ww][threadIdx.x];
            whist[ww][threadIdx.x] = tot;
            tot += c;
        }
    uint32_t total;
    const uint32_t ex = block_excl_scan(threadIdx.x < 256 ? tot : 0u, &total, warp_sums);
    if (threadIdx.x < 256) dbase[threadIdx.x] = ex;
    __syncthreads();
    if (threadIdx.x < 256)
        for (int ww = 0; ww < 32; ++ww) whist[ww][threadIdx.x] += dbase[threadIdx.x];
    __syncthreads();
    for (uint32_t base = b0; base < b1; base += 32) {
        const uint32_t i = base + lane;
        const bool valid = i < b1;
        const uint64_t v = valid ? src[i] : 0ull;
        const uint32_t d = valid ? (uint32_t)((v >> shift) & 255u) : 256u + lane;
        const uint32_t peers = __match_any_sync(0xffffffffu, d);
        const uint32_t rank = __popc(peers & ((1u << lane) - 1u));
        if (valid) dst[whist[w][d] + rank] = v;
        __syncwarp();
        if (valid && lane == __ffs(peers) - 1) whist[w][d] += __popc(peers);
        __syncwarp();
    }
    __syncthreads();
}

// One CTA per half: Y[j] = (sum_{i < l, bit i of j} sw[i] with its low l bits
// cleared) | j, for every j < 2^l, then sorted ascending by an LSD radix sort
// over bits [l, 64) (the low l bits hold the mask and need no ordering).
__global__ void __launch_bounds__(YSORT_THREADS) k_ysort(const HalfJob* __restrict__ hs, int nh) {
    __shared__ uint64_t sw[32];
    __shared__ uint32_t whist[32][256];
    __shared__ uint32_t dbase[256];
    __shared__ uint32_t warp_sums[32];
    const HalfJob J = hs[blockIdx.x];
    const int l = J.l;
    const uint32_t N = 1u << l;
    if (threadIdx.x < J.h) {
        const uint64_t v = J.w[threadIdx.x];
        sw[threadIdx.x] = J.neg ? 0ull - v : v;
    }
    __syncthreads();
    const uint64_t lm = lowmask(l);
    const int passes = N > 1 ? (64 - l + 7) / 8 : 0;
    uint64_t* bufs[2] = {J.ylist, J.ytmp};
    int cur = passes & 1;                       // after `passes` swaps the result is in ylist
    uint64_t* out = bufs[cur];
    enumerate_range(sw, 0, N, [&](uint64_t m, uint64_t key) { out[m] = (key & ~lm) | m; });
    __syncthreads();
    for (int p = 0; p < passes; ++p) {
        lsd_pass(bufs[cur], bufs[cur ^ 1], N, l + 8 * p, whist, dbase, warp_sums);
        cur ^= 1;
    }
}

// Walk the runs x + Y (one per high subset x) of this CTA's share of the
// half and, per bucket, count (COUNT) or write (SCATTER) its records.  In a
// step of 32 elements the lanes are grouped by bucket (__match_any_sync) and
// the group's leader adds the group size to the bucket's counter or reserves
// that many consecutive slots at the bucket's cursor; the order of records
// inside a bucket is irrelevant to the match.
//
// Range mode (at least 16 runs per CTA): the CTA sweeps the buckets in
// ranges of 256.  Because Y is sorted, each run x + Y rotated to its smallest
// key rises, so the records of a run in one bucket range are one contiguous
// stretch; a per-run cursor remembers where the next range starts.  Only the
// cursors of the current range are open, so every bucket's output sectors
// are completed while still in L2.  Warps take runs round robin.
// Piece mode (small halves): warps take pieces of up to 4096 consecutive
// run elements and all buckets stay open (the tables fit in L2 anyway).
constexpr int PIECE = 4096;
constexpr int UNROLL = 4;
constexpr int RANGE = 256;                    // buckets per sweep (at least)
constexpr int RANGE_MAX = 4096;               // buckets per sweep when buckets are many
constexpr int MAX_RUNS_PER_CTA = 1024;
// Piece mode only runs for halves with fewer than 16 runs (h < 20, so at most
// 2^6 buckets); 64 KB covers it and range mode with room to spare.
constexpr int RUNS_SMEM_MAX = 64 * 1024;

struct RunCtx {
    uint64_t lml, lmh, trunc, width, wc, hcap;
    int d1, NB, sh, l, h, neg;
};

// Record r at position p of bucket k (exact layout: p is already absolute).
__device__ __forceinline__ void store_record(const HalfJob& J, uint32_t k, uint32_t p, uint64_t r) {
    if (J.opt_cap) {
        if (p < J.opt_cap) J.tab[(size_t)k * J.opt_cap + p] = r;
        else atomicExch(J.err, 1);                         // region full: redo with the exact layout
    } else {
        J.tab[p] = r;
    }
}

__device__ __forceinline__ void store_halo(const HalfJob& J, const RunCtx& R, uint32_t k, uint64_t Kc, uint64_t m) {
    size_t slot;
    if (J.opt_cap) {
        const uint32_t hp = atomicAdd(&J.hcount[k], 1u);
        if (hp >= J.opt_hcap) { atomicExch(J.err, 1); return; }
        slot = (size_t)k * J.opt_hcap + hp;
    } else {
        const uint32_t hp = atomicAdd(&J.halo_cur[k], 1u);
        if (hp >= R.hcap) return;                           // counted: k_bscan already flagged it
        slot = hp;
    }
    J.halo[2 * slot] = Kc;
    J.halo[2 * slot + 1] = m;
}

// Copy (SCATTER) or count a table-b record into the halo of the neighbouring
// bucket when its coarse window reaches across the bucket edge.
template <bool SCATTER>
__device__ __forceinline__ void halo_check(const HalfJob& J, const RunCtx& R, uint64_t K, uint32_t k, uint64_t m) {
    const uint64_t Kc = K & ~R.trunc;
    const uint64_t off = Kc - ((uint64_t)k << R.sh);
    const uint32_t kl = (k - 1u) & (uint32_t)(R.NB - 1), kh = (k + 1u) & (uint32_t)(R.NB - 1);
    if (SCATTER) {
        if (off < R.wc) store_halo(J, R, kl, Kc, m);
        if (R.width - off <= R.wc) store_halo(J, R, kh, Kc, m);
    } else {
        if (off < R.wc) atomicAdd(&J.halo_cnt[kl], 1u);
        if (R.width - off <= R.wc) atomicAdd(&J.halo_cnt[kh], 1u);
    }
}

// Handle one element (already loaded) of run x: returns its bucket.
template <bool SCATTER>
__device__ __forceinline__ void emit(const HalfJob& J, const RunCtx& R, uint32_t* acc, uint32_t acc_base,
                                     bool valid, uint64_t K, uint32_t k, uint64_t m, uint32_t lane_lt) {
    const int lane = threadIdx.x & 31;
    const uint32_t peers = __match_any_sync(0xffffffffu, valid ? k : 0x80000000u + lane);
    const int leader = __ffs(peers) - 1;
    uint32_t base = 0;
    if (valid && lane == leader)
        base = J.opt_cap ? atomicAdd(&J.bcount[k], (uint32_t)__popc(peers))
                         : atomicAdd(&acc[k - acc_base], (uint32_t)__popc(peers));
    if (SCATTER) {
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) store_record(J, k, base + __popc(peers & lane_lt), ((K << R.d1) & ~R.lmh) | m);
    }
    if (valid && R.neg) {
        const uint64_t Kc = K & ~R.trunc;
        const uint64_t off = Kc - ((uint64_t)k << R.sh);
        const uint32_t kl = (k - 1u) & (uint32_t)(R.NB - 1), kh = (k + 1u) & (uint32_t)(R.NB - 1);
        if (SCATTER) {
            if (off < R.wc) store_halo(J, R, kl, Kc, m);
            if (R.width - off <= R.wc) store_halo(J, R, kh, Kc, m);
        } else {
            if (off < R.wc) atomicAdd(&J.halo_cnt[kl], 1u);
            if (R.width - off <= R.wc) atomicAdd(&J.halo_cnt[kh], 1u);
        }
    }
}

// As emit, for a step whose valid lanes form a prefix (lanes below the first
// set bit of `stops`) with non-decreasing buckets: groups are the maximal
// stretches of equal buckets, found from the boundaries instead of a match.
template <bool SCATTER>
__device__ __forceinline__ void emit_sorted(const HalfJob& J, const RunCtx& R, uint32_t* acc, uint32_t acc_base,
                                            bool valid, uint32_t stops, uint64_t K, uint32_t k, uint64_t m,
                                            uint32_t lane_lt) {
    const int lane = threadIdx.x & 31;
    const uint32_t pk = __shfl_up_sync(0xffffffffu, k, 1);
    const bool head = valid && (lane == 0 || k != pk);
    const uint32_t heads = __ballot_sync(0xffffffffu, head);
    const uint32_t upto = heads & (lane_lt | (1u << lane));            // heads at or below this lane
    const int leader = upto ? 31 - __clz(upto) : 0;
    const uint32_t above = heads & ~(lane_lt | (1u << lane));
    const int first_stop = stops ? __ffs(stops) - 1 : 32;
    const int next_head = above ? __ffs(above) - 1 : 32;
    const int gend = next_head < first_stop ? next_head : first_stop;
    uint32_t base = 0;
    if (head)
        base = J.opt_cap ? atomicAdd(&J.bcount[k], (uint32_t)(gend - lane))
                         : atomicAdd(&acc[k - acc_base], (uint32_t)(gend - lane));
    if (SCATTER) {
        base = __shfl_sync(0xffffffffu, base, leader);
        if (valid) store_record(J, k, base + (uint32_t)(lane - leader), ((K << R.d1) & ~R.lmh) | m);
    }
    if (valid && R.neg) {
        const uint64_t Kc = K & ~R.trunc;
        const uint64_t off = Kc - ((uint64_t)k << R.sh);
        const uint32_t kl = (k - 1u) & (uint32_t)(R.NB - 1), kh = (k + 1u) & (uint32_t)(R.NB - 1);
        if (SCATTER) {
            if (off < R.wc) store_halo(J, R, kl, Kc, m);
            if (R.width - off <= R.wc) store_halo(J, R, kh, Kc, m);
        } else {
            if (off < R.wc) atomicAdd(&J.halo_cnt[kl], 1u);
            if (R.width - off <= R.wc) atomicAdd(&J.halo_cnt[kh], 1u);
        }
    }
}

template <bool SCATTER>
__global__ void __launch_bounds__(PART_THREADS, 2) k_runs(const HalfJob* __restrict__ hs, int nh) {
    extern __shared__ uint32_t dyn[];
    __shared__ uint64_t sw[32];
    const int j = find_last_le(nh, (int)blockIdx.x, [&](int i) { return hs[i].cta_base; });
    const HalfJob J = hs[j];
    const int c = blockIdx.x - J.cta_base;
    RunCtx R;
    R.d1 = J.d1; R.NB = 1 << R.d1; R.sh = 64 - R.d1; R.l = J.l; R.h = J.h; R.neg = J.neg;
    R.lml = lowmask(R.l); R.lmh = lowmask(R.h);
    R.trunc = lowmask(R.h > R.d1 ? R.h - R.d1 : 0);
    R.width = 1ull << R.sh; R.wc = J.wc; R.hcap = J.halo_cap;
    if (threadIdx.x < R.h) {
        const uint64_t v = J.w[threadIdx.x];
        sw[threadIdx.x] = J.neg ? 0ull - v : v;
    }
    const int l = R.l, NB = R.NB;
    const uint32_t N = 1u << l;
    const uint64_t* __restrict__ Y = J.ylist;
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, nwarps = blockDim.x >> 5;
    const uint32_t lt = (1u << lane) - 1u;
    const int hx = R.h - l;
    const bool range_mode = hx >= 4 && ((1 << hx) / J.ctas) >= 16;

    if (!range_mode) {
        uint32_t* acc = dyn;                  // all NB buckets
        for (int b = threadIdx.x; b < NB; b += blockDim.x)
            acc[b] = (SCATTER && !J.opt_cap) ? J.bstart[b] + J.hist[(size_t)c * NB + b] : 0u;
        __syncthreads();
        const uint32_t piece = N < (uint32_t)PIECE ? N : (uint32_t)PIECE;
        const uint32_t per_run = N / piece;
        const uint64_t pieces = (1ull << R.h) / piece;
        const uint64_t p0 = pieces * (uint64_t)c / (uint64_t)J.ctas, p1 = pieces * (uint64_t)(c + 1) / (uint64_t)J.ctas;
        for (uint64_t pc = p0 + warp; pc < p1; pc += nwarps) {
            const uint32_t xi = (uint32_t)(pc / per_run);
            const uint32_t tbeg = (uint32_t)(pc % per_run) * piece;
            uint64_t x = 0;
            for (uint32_t t = xi; t; t &= t - 1) x += sw[l + __ffs(t) - 1];
            const uint64_t xmask = (uint64_t)xi << l;
            for (uint32_t t0 = tbeg; t0 < tbeg + piece; t0 += 32 * UNROLL) {
                uint64_t yv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t t = t0 + 32 * u + lane;
                    yv[u] = t < tbeg + piece ? Y[t] : 0ull;
                }
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t t = t0 + 32 * u + lane;
                    const uint64_t K = x + (yv[u] & ~R.lml);
                    emit<SCATTER>(J, R, acc, 0u, t < tbeg + piece, K, (uint32_t)(K >> R.sh),
                                  xmask | (yv[u] & R.lml), lt);
                }
            }
        }
        if (!SCATTER) {
            __syncthreads();
            uint32_t* out = J.hist + (size_t)c * NB;
            for (int b = threadIdx.x; b < NB; b += blockDim.x) out[b] = acc[b];
        }
        return;
    }

    // ---- range mode
    const uint32_t G = (1u << hx) / (uint32_t)J.ctas;            // runs of this CTA (16..1024)
    const uint32_t x0 = (uint32_t)c * G;
    uint32_t* acc = dyn;                                         // [rw] cursors of the current range
    uint32_t* curx = dyn + RANGE_MAX;                            // [G] next rotated index of each run
    uint32_t* j0s = curx + MAX_RUNS_PER_CTA;                     // [G] rotation (index of the smallest key)
    __syncthreads();
    for (uint32_t g = threadIdx.x; g < G; g += blockDim.x) {
        uint64_t x = 0;
        for (uint32_t t = x0 + g; t; t &= t - 1) x += sw[l + __ffs(t) - 1];
        const uint64_t T = 0ull - x;
        uint32_t lo = 0, hi = N;                                 // first index with (Y & ~lml) >= 2^64 - x
        if (x != 0) {
            while (lo < hi) {
                const uint32_t mid = (lo + hi) >> 1;
                if ((Y[mid] & ~R.lml) >= T) hi = mid; else lo = mid + 1;
            }
        }
        j0s[g] = lo == N ? 0u : lo;
        curx[g] = 0u;
    }
    // sweep width: at least RANGE buckets and about 256 records of each run per sweep
    int rw = RANGE;
    while (rw < RANGE_MAX && (int)(((uint64_t)rw << l) >> R.d1) < 256) rw <<= 1;
    if (rw > NB) rw = NB;
    const int nrange = NB / rw;
    for (int r = 0; r < nrange; ++r) {
        const uint32_t k0 = (uint32_t)r * rw, kend = k0 + rw;
        __syncthreads();
        for (int b = threadIdx.x; b < rw; b += blockDim.x)
            acc[b] = (SCATTER && !J.opt_cap) ? J.bstart[k0 + b] + J.hist[(size_t)c * NB + k0 + b] : 0u;
        __syncthreads();
        for (uint32_t g = warp; g < G; g += nwarps) {
            const uint32_t xi = x0 + g;
            uint64_t x = 0;
            for (uint32_t t = xi; t; t &= t - 1) x += sw[l + __ffs(t) - 1];
            const uint64_t xmask = (uint64_t)xi << l;
            const uint32_t j0 = j0s[g];
            uint32_t t0 = curx[g];
            bool done = t0 >= N;
            while (!done) {
                // 1. load UNROLL steps, compute keys, buckets and stop lanes
                uint64_t Kv[UNROLL], mv[UNROLL];
                uint32_t kv[UNROLL], stv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t t = t0 + 32 * u + lane;
                    const uint64_t y = t < N ? Y[(j0 + t) & (N - 1)] : 0ull;
                    Kv[u] = x + (y & ~R.lml);
                    mv[u] = xmask | (y & R.lml);
                    kv[u] = (uint32_t)(Kv[u] >> R.sh);
                }
                int nsteps = UNROLL;
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    const uint32_t t = t0 + 32 * u + lane;
                    stv[u] = __ballot_sync(0xffffffffu, t >= N || kv[u] >= kend);   // keys rise along the run
                    if (stv[u] && nsteps == UNROLL) nsteps = u + 1;
                }
                // 2. one reservation per bucket group, all steps' atomics in flight together
                uint32_t bv[UNROLL];
                int lv[UNROLL];
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    bv[u] = 0; lv[u] = 0;
                    if (u >= nsteps) continue;
                    const int first_stop = stv[u] ? __ffs(stv[u]) - 1 : 32;
                    const bool valid = lane < first_stop;
                    const uint32_t pk = __shfl_up_sync(0xffffffffu, kv[u], 1);
                    const bool head = valid && (lane == 0 || kv[u] != pk);
                    const uint32_t heads = __ballot_sync(0xffffffffu, head);
                    const uint32_t upto = heads & (lt | (1u << lane));
                    lv[u] = upto ? 31 - __clz(upto) : 0;
                    const uint32_t above = heads & ~(lt | (1u << lane));
                    const int next_head = above ? __ffs(above) - 1 : 32;
                    const int gend = next_head < first_stop ? next_head : first_stop;
                    if (head)
                        bv[u] = J.opt_cap ? atomicAdd(&J.bcount[kv[u]], (uint32_t)(gend - lane))
                                          : atomicAdd(&acc[kv[u] - k0], (uint32_t)(gend - lane));
                }
                // 3. positions, records, halo
#pragma unroll
                for (int u = 0; u < UNROLL; ++u) {
                    if (u >= nsteps) continue;
                    const int first_stop = stv[u] ? __ffs(stv[u]) - 1 : 32;
                    const bool valid = lane < first_stop;
                    if (SCATTER) {
                        const uint32_t base = __shfl_sync(0xffffffffu, bv[u], lv[u]);
                        if (valid) store_record(J, kv[u], base + (uint32_t)(lane - lv[u]), ((Kv[u] << R.d1) & ~R.lmh) | mv[u]);
                    }
                    if (valid && R.neg) halo_check<SCATTER>(J, R, Kv[u], kv[u], mv[u]);
                }
                if (stv[nsteps - 1]) {
                    done = true;
                    t0 = t0 + 32 * (nsteps - 1) + (__ffs(stv[nsteps - 1]) - 1);
                } else {
                    t0 += 32 * UNROLL;
                }
            }
            if (lane == 0) curx[g] = t0;
        }
        __syncthreads();
        if (!SCATTER)
            for (int b = threadIdx.x; b < rw; b += blockDim.x) J.hist[(size_t)c * NB + k0 + b] = acc[b];
    }
}

__global__ void __launch_bounds__(256) k_colscan(const HalfJob* __restrict__ hs, int nh) {
    const int j = find_last_le(nh, (int)blockIdx.x, [&](int i) { return hs[i].scan_base; });
    const HalfJob J = hs[j];
    const int NB = 1 << J.d1;
    const int b = (blockIdx.x - J.scan_base) * blockDim.x + threadIdx.x;
    if (b >= NB) return;
    uint32_t run = 0;
    for (int c = 0; c < J.ctas; ++c) {
        uint32_t* p = J.hist + (size_t)c * NB + b;
        const uint32_t t = *p;
        *p = run;
        run += t;
    }
    J.bstart[b] = run;
}

__global__ void __launch_bounds__(1024) k_bscan(const HalfJob* __restrict__ hs, int nh) {
    __shared__ uint32_t warp_sums[32];
    const HalfJob J = hs[blockIdx.x];
    const int NB = 1 << J.d1;
    block_scan_array(J.bstart, NB, true, warp_sums);
    if (J.neg) {
        __syncthreads();
        block_scan_array(J.halo_cnt, NB, true, warp_sums);
        __syncthreads();
        for (int b = threadIdx.x; b < NB; b += blockDim.x) J.halo_cur[b] = J.halo_cnt[b];
        if (threadIdx.x == 0 && (uint64_t)J.halo_cnt[NB] > J.halo_cap) atomicExch(J.err, 1);
    }
}

// ---------------------------------------------------------------- digit 2 + K-e
__device__ __forceinline__ uint64_t subset_sum(const uint64_t* w, uint64_t m) {
    uint64_t s = 0;
    for (; m; m &= m - 1) s += w[__ffsll((long long)m) - 1];
    return s;
}

__global__ void __launch_bounds__(JOIN_THREADS, 2) k_join(const ProbJob* __restrict__ ps, int np) {
    extern __shared__ uint64_t smem[];
    uint64_t* As = smem;
    uint32_t* off = reinterpret_cast<uint32_t*>(As + JOIN_CAP);
    __shared__ uint64_t wa[32], w2a[32], wb[32], w2b[32];
    __shared__ uint32_t warp_sums[32];
    const int j = find_last_le(np, (int)blockIdx.x, [&](int i) { return ps[i].join_base; });
    const ProbJob& P = ps[j];
    const int k = blockIdx.x - P.join_base;
    const int n_a = P.n_a, n_b = P.n_b, d1 = P.d1;
    if (threadIdx.x < n_a) { wa[threadIdx.x] = P.w_a[threadIdx.x]; w2a[threadIdx.x] = P.w2_a[threadIdx.x]; }
    if (threadIdx.x < n_b) { wb[threadIdx.x] = P.w_b[threadIdx.x]; w2b[threadIdx.x] = P.w2_b[threadIdx.x]; }
    const int sh = 64 - d1;
    const int subsh = sh - SUB_BITS;
    const uint64_t lo_k = (uint64_t)k << sh;
    const long long width = (long long)(1ull << sh);
    const uint64_t la = lowmask(n_a), lb = lowmask(n_b);
    uint64_t a0, a1, b0, b1, h0, h1;
    if (P.A.opt_cap) {
        a0 = (uint64_t)k * P.A.opt_cap; a1 = a0 + min(P.A.bcount[k], P.A.opt_cap);
        b0 = (uint64_t)k * P.B.opt_cap; b1 = b0 + min(P.B.bcount[k], P.B.opt_cap);
        h0 = (uint64_t)k * P.B.opt_hcap; h1 = h0 + min(P.B.hcount[k], P.B.opt_hcap);
    } else {
        const uint64_t hcap = P.B.halo_cap;
        a0 = P.A.bstart[k]; a1 = P.A.bstart[k + 1];
        b0 = P.B.bstart[k]; b1 = P.B.bstart[k + 1];
        h0 = min((uint64_t)P.B.halo_cnt[k], hcap);
        h1 = min((uint64_t)P.B.halo_cnt[k + 1], hcap);
    }
    const uint32_t nbn = (uint32_t)(b1 - b0), nbt = nbn + (uint32_t)(h1 - h0);
    const uint64_t Wc = P.Wc, W = P.W, W2 = P.W2;
    const uint64_t* __restrict__ tabA = P.A.tab;
    const uint64_t* __restrict__ tabB = P.B.tab;
    const uint64_t* __restrict__ halo = P.B.halo;
    unsigned long long n_coarse = 0, n_pre = 0;
    __syncthreads();
    constexpr int U = 4;                       // independent loads in flight per thread
    const uint32_t stride = blockDim.x * U;
    for (uint64_t cs = a0; cs < a1; cs += JOIN_CAP) {
        const uint32_t m = (uint32_t)min((uint64_t)JOIN_CAP, a1 - cs);
        for (int s = threadIdx.x; s < pad32(1 << SUB_BITS); s += blockDim.x) off[s] = 0u;
        __syncthreads();
        // digit 2 = the top 13 bits of the record (key bits below the bucket's d1 bits)
        for (uint32_t i0 = threadIdx.x; i0 < m; i0 += stride) {
            uint64_t r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) r[u] = i0 + u * blockDim.x < m ? tabA[cs + i0 + u * blockDim.x] : 0ull;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + u * blockDim.x < m) atomicAdd(&off[pad32((int)(r[u] >> (64 - SUB_BITS)))], 1u);
        }
        __syncthreads();
        block_scan_padded(off, 1 << SUB_BITS, warp_sums);
        __syncthreads();
        for (uint32_t i0 = threadIdx.x; i0 < m; i0 += stride) {
            uint64_t r[U];
#pragma unroll
            for (int u = 0; u < U; ++u) r[u] = i0 + u * blockDim.x < m ? tabA[cs + i0 + u * blockDim.x] : 0ull;
#pragma unroll
            for (int u = 0; u < U; ++u)
                if (i0 + u * blockDim.x < m) As[atomicAdd(&off[pad32((int)(r[u] >> (64 - SUB_BITS)))], 1u)] = r[u];
        }
        __syncthreads();
        // Records of one bucket hold (key << d1) with their low bits cleared,
        // so |Ka - Kb| < Wc is |ra - rb| < Wc << d1 on the masked records.
        const uint64_t Wd = Wc << d1;
        auto hit = [&](uint64_t ra, uint64_t mb) {
            ++n_coarse;
            const uint64_t ma = ra & la;
            const uint64_t v = subset_sum(wa, ma) + subset_sum(wb, mb);
            if (circ_dist(v) <= W) {
                ++n_pre;
                const uint64_t t2 = subset_sum(w2a, ma) + subset_sum(w2b, mb);
                if (circ_dist(t2) <= W2) {
                    if (ma == 0 && mb == 0) {
                        P.ctr[3] = 1ull;
                    } else {
                        const unsigned long long idx = atomicAdd(&P.ctr[2], 1ull);
                        if (idx < P.cap) P.cand[idx] = ma | (mb << n_a);
                    }
                }
            }
        };
        for (uint32_t t0 = threadIdx.x; t0 < nbn; t0 += stride) {
            uint64_t rb[U];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const uint32_t t = t0 + u * blockDim.x;
                rb[u] = t < nbn ? tabB[b0 + t] : 0ull;
            }
#pragma unroll
            for (int u = 0; u < U; ++u) {
                if (t0 + u * blockDim.x >= nbn) continue;
                const uint64_t rkb = rb[u] & ~lb, mb = rb[u] & lb;
                const uint64_t lo = rkb > Wd - 1 ? rkb - (Wd - 1) : 0ull;
                const uint64_t hi = rkb < ~0ull - (Wd - 1) ? rkb + (Wd - 1) : ~0ull;
                const int s_lo = (int)(lo >> (64 - SUB_BITS)), s_hi = (int)(hi >> (64 - SUB_BITS));
                const uint32_t p0 = s_lo ? off[pad32(s_lo - 1)] : 0u, p1 = off[pad32(s_hi)];
                for (uint32_t p = p0; p < p1; ++p) {
                    const uint64_t ra = As[p];
                    const long long diff = (long long)((ra & ~la) - rkb);
                    if (diff > -(long long)Wd && diff < (long long)Wd) hit(ra, mb);
                }
            }
        }
        // halo records (from the neighbouring buckets): full coarse keys
        for (uint32_t t = nbn + threadIdx.x; t < nbt; t += blockDim.x) {
            const size_t hi2 = 2 * (size_t)(h0 + (t - nbn));
            const uint64_t Kb = halo[hi2], mb = halo[hi2 + 1];
            long long dlo = (long long)(Kb - Wc + 1ull - lo_k);
            long long dhi = (long long)(Kb + Wc - 1ull - lo_k);
            if (dhi < 0 || dlo >= width) continue;
            if (dlo < 0) dlo = 0;
            if (dhi > width - 1) dhi = width - 1;
            const int s_lo = (int)(dlo >> subsh), s_hi = (int)(dhi >> subsh);
            const uint32_t p0 = s_lo ? off[pad32(s_lo - 1)] : 0u, p1 = off[pad32(s_hi)];
            for (uint32_t p = p0; p < p1; ++p) {
                const uint64_t ra = As[p];
                const uint64_t Ka = lo_k | ((ra & ~la) >> d1);
                const long long diff = (long long)(Ka - Kb);
                if (diff > -(long long)Wc && diff < (long long)Wc) hit(ra, mb);
            }
        }
        __syncthreads();
    }
    if (n_coarse) atomicAdd(&P.ctr[0], n_coarse);
    if (n_pre) atomicAdd(&P.ctr[1], n_pre);
}

// ---------------------------------------------------------------- fused small match
// One CTA per problem with n_b <= 13: the 2^n_a table-a keys are enumerated
// (Gray code) and counting-sorted by their top 13 bits into shared memory;
// the 2^n_b table-b keys are enumerated on the fly and probe the circular
// window directly.  Records are (key & ~(2^n_a - 1)) | mask, so the coarse
// window is W + 2^n_a and every coarse hit is re-checked exactly.  No global
// tables, one launch for all small problems of a batch.
__global__ void __launch_bounds__(SMALL_THREADS, 2) k_small(const SmallJob* __restrict__ js, int np) {
    extern __shared__ uint64_t smem[];
    uint64_t* As = smem;                                       // 2^13 records
    uint32_t* off = reinterpret_cast<uint32_t*>(As + (1 << SMALL_MAX_H));
    __shared__ uint64_t wa[32], w2a[32], wb[32], w2b[32], nwb[32];
    __shared__ uint32_t warp_sums[32];
    const SmallJob& P = js[blockIdx.x];
    const int n_a = P.n_a, n_b = P.n_b;
    if (threadIdx.x < n_a) { wa[threadIdx.x] = P.w_a[threadIdx.x]; w2a[threadIdx.x] = P.w2_a[threadIdx.x]; }
    if (threadIdx.x < n_b) {
        wb[threadIdx.x] = P.w_b[threadIdx.x];
        w2b[threadIdx.x] = P.w2_b[threadIdx.x];
        nwb[threadIdx.x] = 0ull - P.w_b[threadIdx.x];
    }
    for (int s = threadIdx.x; s < pad32(1 << SUB_BITS); s += blockDim.x) off[s] = 0u;
    __syncthreads();
    const uint64_t la = lowmask(n_a), lb = lowmask(n_b);
    const uint64_t Na = 1ull << n_a, Nb = 1ull << n_b;
    const uint64_t W = P.W, W2 = P.W2, Wc = W + (1ull << n_a);
    const int top = 64 - SUB_BITS;
    enumerate_range(wa, 0, Na, [&](uint64_t m, uint64_t key) {
        atomicAdd(&off[pad32((int)(key >> top))], 1u);
    });
    __syncthreads();
    block_scan_padded(off, 1 << SUB_BITS, warp_sums);
    __syncthreads();
    enumerate_range(wa, 0, Na, [&](uint64_t m, uint64_t key) {
        As[atomicAdd(&off[pad32((int)(key >> top))], 1u)] = (key & ~la) | m;
    });
    __syncthreads();
    unsigned long long n_coarse = 0, n_pre = 0;
    auto probe_range = [&](int s0, int s1, uint64_t Kb, uint64_t mb) {
        const uint32_t p0 = s0 ? off[pad32(s0 - 1)] : 0u, p1 = off[pad32(s1)];
        for (uint32_t p = p0; p < p1; ++p) {
            const uint64_t ra = As[p];
            const long long diff = (long long)((ra & ~la) - Kb);
            if (diff > -(long long)Wc && diff < (long long)Wc) {
                ++n_coarse;
                const uint64_t ma = ra & la;
                const uint64_t v = subset_sum(wa, ma) + subset_sum(wb, mb);
                if (circ_dist(v) <= W) {
                    ++n_pre;
                    const uint64_t t2 = subset_sum(w2a, ma) + subset_sum(w2b, mb);
                    if (circ_dist(t2) <= W2) {
                        if (ma == 0 && mb == 0) {
                            P.ctr[3] = 1ull;
                        } else {
                            const unsigned long long idx = atomicAdd(&P.ctr[2], 1ull);
                            if (idx < P.cap) P.cand[idx] = ma | (mb << n_a);
                        }
                    }
                }
            }
        }
    };
    enumerate_range(nwb, 0, Nb, [&](uint64_t mb, uint64_t Kb) {
        const uint64_t lo = Kb - Wc + 1ull, hi = Kb + Wc - 1ull;
        const int s_lo = (int)(lo >> top), s_hi = (int)(hi >> top);
        if (lo <= hi) {
            probe_range(s_lo, s_hi, Kb, mb);
        } else {                                               // the window wraps past 2^64
            probe_range(s_lo, (1 << SUB_BITS) - 1, Kb, mb);
            probe_range(0, s_hi, Kb, mb);
        }
    });
    if (n_coarse) atomicAdd(&P.ctr[0], n_coarse);
    if (n_pre) atomicAdd(&P.ctr[1], n_pre);
}

static const size_t SMALL_SMEM = ((size_t)1 << SMALL_MAX_H) * 8 + (size_t)pad32(1 << SUB_BITS) * 4;
static PerDeviceOnce g_small_attr;

cudaError_t small_attrs() {
    return g_small_attr.run([] {
        return cudaFuncSetAttribute(k_small, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)SMALL_SMEM);
    });
}

cudaError_t small_issue(const SmallJob* dev_jobs, int np, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    k_small<<<np, SMALL_THREADS, SMALL_SMEM, s>>>(dev_jobs, np);
    return cudaGetLastError();
}

cudaError_t run_small(const SmallJob* jobs, int np, SmallJob* dev_jobs, cudaStream_t s) {
    if (np <= 0) return cudaSuccess;
    cudaError_t e = small_attrs();
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dev_jobs, jobs, sizeof(SmallJob) * np, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    return small_issue(dev_jobs, np, s);
}

// ---------------------------------------------------------------- host side
static size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

static uint64_t default_halo_cap(int n_b, int d1, uint64_t wc) {
    const uint64_t Nb = 1ull << n_b;
    const double frac = 2.0 * (double)wc / (double)(1ull << (64 - d1));
    const double want = frac * 1.5 * (double)Nb + 4096.0;
    return want >= (double)Nb ? Nb : (uint64_t)want;
}

size_t match_bytes(const MatchGeom& g) {
    if (g.splat || g.prune) return g.bytes;
    if (g.fused) return mitm_half_bytes(g.l_a) + mitm_half_bytes(g.l_b) + align256(mitm_hit_cap(g) * 8);
    const size_t NB = (size_t)1 << g.d1;
    size_t b = 0;
    b += 2 * align256(((size_t)1 << g.l_a) * 8);
    b += 2 * align256(((size_t)1 << g.l_b) * 8);
    if (g.optimistic) {
        b += align256(NB * g.cap_a * 8) + align256(NB * g.cap_b * 8);
        b += align256(NB * 4) * 3 + align256(NB * g.hcap_per * 16);
        return b;
    }
    b += align256(((size_t)1 << g.n_a) * 8);
    b += align256(((size_t)1 << g.n_b) * 8);
    b += align256((size_t)g.ctas_a * NB * 4);
    b += align256((size_t)g.ctas_b * NB * 4);
    b += 2 * align256((NB + 1) * 4);
    b += align256((NB + 1) * 4) + align256(NB * 4);
    b += align256((size_t)g.hcap * 16);
    return b;
}

// CTAs of a half: range mode (16 .. 1024 runs per CTA) when it has at least
// 16 runs, else at most one CTA per piece of up to 4096 run elements.
static int clamp_ctas(int h, int l, int want) {
    const int hx = h - l;
    if (hx >= 4) {
        int lo = hx > 10 ? 1 << (hx - 10) : 1, hi = 1 << (hx - 4);
        int c = want < lo ? lo : (want > hi ? hi : want);
        return c;
    }
    const int pieces = h > 12 ? 1 << (h - 12) : 1;
    return want < pieces ? (want < 1 ? 1 : want) : pieces;
}

bool match_geometry(int n_a, int n_b, uint64_t W, int ctas_a, int ctas_b, MatchGeom* g, bool optimistic,
                    const TuneParams* tp, int fuse) {
    if (n_a < 0 || n_b < n_a || n_b > 32) return false;
    g->splat = false;
    g->prune = false;
    if (optimistic && fuse == FUSE_SPLAT) {
        if (splat_geometry(n_a, n_b, g)) return true;
        fuse = FUSE_AUTO;
    }
    if (optimistic && fuse == FUSE_PRUNE) {
        if (prune_geometry(n_a, n_b, g)) return true;
        fuse = FUSE_AUTO;
    }
    if (optimistic && (fuse == FUSE_ALWAYS || (fuse == FUSE_AUTO && n_a >= FUSED_MIN_NA))) {
        if (mitm_geometry(n_a, n_b, W, g, tp)) return true;
        if (fuse == FUSE_ALWAYS) return false;
    }
    g->fused = false;
    g->nbl = g->slab = g->wf = 0;
    const TuneParams dflt;
    if (!tp) tp = &dflt;
    const int lm = tp->l_max < 10 ? 10 : (tp->l_max > 18 ? 18 : tp->l_max);
    const int l_a = n_a < lm ? n_a : lm, l_b = n_b < lm ? n_b : lm;
    int d1 = n_a - tp->d1_off;
    if (d1 < 2) d1 = 2;
    if (d1 > MAX_D1) d1 = MAX_D1;
    uint64_t wc = 0;
    for (; d1 >= 2; --d1) {
        // coarse keys lose < 2^l (truncated low-list sums) + 2^tr (record truncation)
        const int tr = n_b > d1 ? n_b - d1 : 0;
        wc = W + (1ull << l_b) + (1ull << tr);
        if (wc < W) continue;                                  // overflow
        if (wc < (1ull << (64 - d1)) / 4) break;
    }
    if (d1 < 2) return false;
    g->n_a = n_a; g->n_b = n_b; g->d1 = d1; g->wc = wc;
    g->l_a = l_a; g->l_b = l_b;
    g->ctas_a = clamp_ctas(n_a, l_a, ctas_a);
    g->ctas_b = clamp_ctas(n_b, l_b, ctas_b);
    g->hcap = default_halo_cap(n_b, d1, wc);
    // optimistic layout: 25 % + 64 slack per bucket over the mean count (keys of
    // random polynomials spread evenly; clustered keys overflow and are redone
    // with the exact layout)
    g->optimistic = optimistic && d1 >= 2;
    const uint64_t ea = (1ull << n_a) >> d1, eb = (1ull << n_b) >> d1;
    g->cap_a = (uint32_t)((ea + ea / 4 + 64 + 3) & ~3ull);
    g->cap_b = (uint32_t)((eb + eb / 4 + 64 + 3) & ~3ull);
    const double halo_mean = 2.0 * (double)wc / (double)(1ull << (64 - d1)) * (double)eb;
    g->hcap_per = (uint32_t)(8.0 + 4.0 * halo_mean);
    g->bytes = match_bytes(*g);
    return true;
}

void match_layout(const MatchGeom& g, char* ws, ProbJob* pj) {
    const size_t NB = (size_t)1 << g.d1;
    char* p = ws;
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    HalfJob& A = pj->A;
    HalfJob& B = pj->B;
    pj->splat = 0;
    pj->gamma = nullptr;
    pj->prune = 0;
    if (g.splat) {
        splat_layout(g, ws, pj);
        return;
    }
    if (g.prune) {
        pj->prune = 1;
        pj->fused = 0;
        pj->n_a = g.n_a; pj->n_b = g.n_b;
        return;
    }
    pj->fused = g.fused ? 1 : 0;
    pj->nbl = g.nbl; pj->slab = g.slab; pj->wf = g.wf;
    A.kb1 = B.kb1 = nullptr; A.ysplit = B.ysplit = nullptr;
    pj->hits = nullptr; pj->hcap = 0;
    if (g.fused) {
        mitm_layout_half(g.l_a, p, &A);
        mitm_layout_half(g.l_b, p, &B);
        pj->hcap = mitm_hit_cap(g);
        pj->hits = (uint64_t*)take(pj->hcap * 8);
        A.l = g.l_a; B.l = g.l_b;
        A.h = g.n_a; B.h = g.n_b;
        A.neg = 0; B.neg = 1;
        A.d1 = B.d1 = g.d1;
        A.ctas = B.ctas = 0;
        A.wc = B.wc = g.wc;
        pj->n_a = g.n_a; pj->n_b = g.n_b; pj->d1 = g.d1; pj->Wc = g.wc;
        A.hist = B.hist = nullptr; A.bstart = B.bstart = nullptr; A.tab = B.tab = nullptr;
        A.halo_cnt = B.halo_cnt = nullptr; A.halo_cur = B.halo_cur = nullptr; A.halo = B.halo = nullptr;
        A.halo_cap = B.halo_cap = 0; A.opt_cap = B.opt_cap = 0; A.opt_hcap = B.opt_hcap = 0;
        A.bcount = B.bcount = nullptr; A.hcount = B.hcount = nullptr;
        return;
    }
    A.ylist = (uint64_t*)take(((size_t)1 << g.l_a) * 8);
    A.ytmp = (uint64_t*)take(((size_t)1 << g.l_a) * 8);
    B.ylist = (uint64_t*)take(((size_t)1 << g.l_b) * 8);
    B.ytmp = (uint64_t*)take(((size_t)1 << g.l_b) * 8);
    A.l = g.l_a; B.l = g.l_b;
    A.h = g.n_a; B.h = g.n_b;
    A.neg = 0; B.neg = 1;
    A.d1 = B.d1 = g.d1;
    A.ctas = g.ctas_a; B.ctas = g.ctas_b;
    A.wc = B.wc = g.wc;
    pj->n_a = g.n_a; pj->n_b = g.n_b; pj->d1 = g.d1; pj->Wc = g.wc;
    A.halo_cnt = nullptr; A.halo_cur = nullptr; A.halo = nullptr; A.halo_cap = 0;
    A.hcount = nullptr; A.opt_hcap = 0;
    if (g.optimistic) {
        A.opt_cap = g.cap_a; B.opt_cap = g.cap_b; B.opt_hcap = g.hcap_per;
        A.tab = (uint64_t*)take(NB * g.cap_a * 8);
        B.tab = (uint64_t*)take(NB * g.cap_b * 8);
        A.bcount = (uint32_t*)take(NB * 4);
        B.bcount = (uint32_t*)take(NB * 4);
        B.hcount = (uint32_t*)take(NB * 4);
        B.halo = (uint64_t*)take(NB * g.hcap_per * 16);
        B.halo_cap = 0;
        A.hist = B.hist = nullptr; A.bstart = B.bstart = nullptr;
        B.halo_cnt = nullptr; B.halo_cur = nullptr;
        return;
    }
    A.opt_cap = B.opt_cap = 0; B.opt_hcap = 0;
    A.bcount = B.bcount = nullptr; B.hcount = nullptr;
    A.tab = (uint64_t*)take(((size_t)1 << g.n_a) * 8);
    B.tab = (uint64_t*)take(((size_t)1 << g.n_b) * 8);
    A.hist = (uint32_t*)take((size_t)g.ctas_a * NB * 4);
    B.hist = (uint32_t*)take((size_t)g.ctas_b * NB * 4);
    A.bstart = (uint32_t*)take((NB + 1) * 4);
    B.bstart = (uint32_t*)take((NB + 1) * 4);
    B.halo_cnt = (uint32_t*)take((NB + 1) * 4);
    B.halo_cur = (uint32_t*)take(NB * 4);
    B.halo_cap = g.hcap;
    B.halo = (uint64_t*)take((size_t)g.hcap * 16);
}

// Assign grid bases for a set of problems; fills halves[2*np].
struct MatchGrid { int part_ctas, scan_ctas, join_ctas, nb_max, nb_small; };

static bool is_range_mode(const HalfJob& h) {
    const int hx = h.h - h.l;
    return hx >= 4 && ((1 << hx) / h.ctas) >= 16;
}

static MatchGrid assign_bases(ProbJob* jobs, int np, HalfJob* halves) {
    MatchGrid g{0, 0, 0, 0, 0};
    for (int i = 0; i < np; ++i) {
        ProbJob& P = jobs[i];
        const int NB = 1 << P.d1;
        HalfJob* hh[2] = {&P.A, &P.B};
        for (int t = 0; t < 2; ++t) {
            hh[t]->cta_base = g.part_ctas;
            g.part_ctas += hh[t]->ctas;
            hh[t]->scan_base = g.scan_ctas;
            g.scan_ctas += (NB + 255) / 256;
            if (!is_range_mode(*hh[t]) && NB > g.nb_small) g.nb_small = NB;
            halves[2 * i + t] = *hh[t];
        }
        P.join_base = g.join_ctas;
        g.join_ctas += NB;
        if (NB > g.nb_max) g.nb_max = NB;
    }
    return g;
}

static PerDeviceOnce g_attr_set;
static const size_t JOIN_SMEM = (size_t)JOIN_CAP * 8 + ((size_t)1 << SUB_BITS) * 4 + ((size_t)1 << SUB_BITS) / 32 * 4;

// Upload jobs (from host memory that stays valid until the copies finish:
// pageable memory is staged before cudaMemcpyAsync returns) and launch.
cudaError_t run_match(ProbJob* jobs, int np, ProbJob* dev_jobs, HalfJob* dev_halves,
                      HalfJob* host_halves, cudaStream_t s, cudaEvent_t ev_count, cudaEvent_t ev_scatter,
                      int* launches) {
    {
        cudaError_t e = g_attr_set.run([] {
            cudaError_t r = cudaFuncSetAttribute(k_join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JOIN_SMEM);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(k_runs<false>, cudaFuncAttributeMaxDynamicSharedMemorySize, RUNS_SMEM_MAX);
            if (r == cudaSuccess)
                r = cudaFuncSetAttribute(k_runs<true>, cudaFuncAttributeMaxDynamicSharedMemorySize, RUNS_SMEM_MAX);
            return r;
        });
        if (e != cudaSuccess) return e;
    }
    // table problems first (compacted to the front of a copy), fused ones after
    std::vector<ProbJob> T;
    std::vector<const ProbJob*> F, Sp, Pr;
    for (int i = 0; i < np; ++i) {
        if (jobs[i].prune) Pr.push_back(&jobs[i]);
        else if (jobs[i].splat) Sp.push_back(&jobs[i]);
        else if (jobs[i].fused) F.push_back(&jobs[i]);
        else T.push_back(jobs[i]);
    }
    const int nT = (int)T.size(), nF = (int)F.size(), nS = (int)Sp.size(), nP = (int)Pr.size();
    int nl = 0;
    cudaError_t e = cudaSuccess;
    if (nT) {
        MatchGrid g = assign_bases(T.data(), nT, host_halves);
        e = cudaMemcpyAsync(dev_halves, host_halves, sizeof(HalfJob) * 2 * nT, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        e = cudaMemcpyAsync(dev_jobs, T.data(), sizeof(ProbJob) * nT, cudaMemcpyHostToDevice, s);
        if (e != cudaSuccess) return e;
        size_t psmem = (size_t)(RANGE_MAX + 2 * MAX_RUNS_PER_CTA) * 4;
        if ((size_t)g.nb_small * 4 > psmem) psmem = (size_t)g.nb_small * 4;
        if (psmem > (size_t)RUNS_SMEM_MAX) return cudaErrorInvalidConfiguration;
        k_ysort<<<2 * nT, YSORT_THREADS, 0, s>>>(dev_halves, 2 * nT);
        ++nl;
        if (!T[0].A.opt_cap) {
            k_runs<false><<<g.part_ctas, PART_THREADS, psmem, s>>>(dev_halves, 2 * nT);
            k_colscan<<<g.scan_ctas, 256, 0, s>>>(dev_halves, 2 * nT);
            k_bscan<<<2 * nT, 1024, 0, s>>>(dev_halves, 2 * nT);
            nl += 3;
        }
        if (ev_count) cudaEventRecord(ev_count, s);
        k_runs<true><<<g.part_ctas, PART_THREADS, psmem, s>>>(dev_halves, 2 * nT);
        if (ev_scatter) cudaEventRecord(ev_scatter, s);
        k_join<<<g.join_ctas, JOIN_THREADS, JOIN_SMEM, s>>>(dev_jobs, nT);
        nl += 2;
        e = cudaGetLastError();
        if (e != cudaSuccess) return e;
    }
    if (nF) {
        e = run_mitm(F.data(), nF, dev_jobs + nT, dev_halves + 2 * nT, s, nT ? nullptr : ev_count,
                     nT ? nullptr : ev_scatter);
        nl += mitm_launches(F.data(), nF);
        if (e != cudaSuccess) return e;
    } else if (!nT) {
        if (ev_count) cudaEventRecord(ev_count, s);
        if (ev_scatter) cudaEventRecord(ev_scatter, s);
    }
    if (nS) {
        e = run_splat(Sp.data(), nS, dev_jobs + nT + nF, s);
        nl += 2;
        if (e != cudaSuccess) return e;
    }
    if (nP) {
        e = run_prune(Pr.data(), nP, dev_jobs + nT + nF + nS, s);
        nl += 1;
    }
    if (launches) *launches = nl;
    return e;
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_enumerate(const uint64_t* w, int h, uint64_t* keys, void* stream) {
    if (!w || !keys || h < 0 || h > 32 || (((uintptr_t)keys) & 15)) return RFR_E_INVALID;
    if (h == 0) {
        return cudaMemsetAsync(keys, 0, 8, (cudaStream_t)stream) == cudaSuccess ? RFR_OK : RFR_E_CUDA;
    }
    int blocks;
    if (h < 6) blocks = 1;
    else {
        const uint64_t nhigh = 1ull << (h - 6);          // warp steps
        uint64_t warps = nhigh < 148ull * 64 ? nhigh : 148ull * 64;
        blocks = (int)((warps + 7) / 8);
    }
    k_enum_plain<<<blocks, 256, 0, (cudaStream_t)stream>>>(w, h, keys);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}

static int stage_ctas(int h) {
    int c = h > 20 ? 1 << (h - 20) : 1;
    return c > 256 ? 256 : c;
}

// Stage workspace: job structs, then one problem's buffers with a halo large
// enough for every record of table b (so no window can overflow it).
static bool stage_geom(int n_a, int n_b, uint64_t W, MatchGeom* g, bool optimistic, int fuse = FUSE_AUTO) {
    if (!match_geometry(n_a, n_b, W, stage_ctas(n_a), stage_ctas(n_b), g, optimistic, nullptr, fuse)) return false;
    g->hcap = 1ull << n_b;
    g->bytes = match_bytes(*g);
    return true;
}

extern "C" size_t rfr_stage_match_workspace(int n_a, int n_b) {
    MatchGeom g, go, gf;
    if (!stage_geom(n_a, n_b, 0, &g, false)) return 0;
    if (stage_geom(n_a, n_b, 0, &go, true) && go.bytes > g.bytes) g.bytes = go.bytes;
    if (stage_geom(n_a, n_b, 0, &gf, true, FUSE_ALWAYS)) {
        // room for the fused match's fingerprint hits: up to 2^20 pairs (more hits, at
        // very wide windows, report counters[4] unless the caller passes more workspace)
        const int e = n_a + n_b < 20 ? n_a + n_b : 20;
        const size_t fb = gf.bytes + ((size_t)8 << e);
        if (fb > g.bytes) g.bytes = fb;
    }
    // the bucket count only shrinks for wider windows; budget for d1 = MAX_D1 histograms
    const size_t hist_extra = ((size_t)stage_ctas(n_a) + stage_ctas(n_b)) * ((size_t)1 << MAX_D1) * 4 + 8 * 4096;
    return g.bytes + hist_extra + 2048;
}

extern "C" size_t rfr_stage_match_fused_workspace(int n_a, int n_b) {
    MatchGeom gf;
    if (!stage_geom(n_a, n_b, 0, &gf, true, FUSE_ALWAYS)) return 0;
    const int e = n_a + n_b < 20 ? n_a + n_b : 20;
    return gf.bytes + ((size_t)8 << e) + 2048;
}

static int stage_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                       const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                       uint64_t window, uint64_t window2,
                       void* workspace, size_t workspace_bytes,
                       uint64_t* cand, uint64_t cap, uint64_t* counters, void* stream, bool optimistic,
                       int fuse = FUSE_AUTO) {
    if (n_a < 0 || n_b < n_a || n_b > 32 || !workspace || !counters || (!cand && cap)) return RFR_E_INVALID;
    if ((n_a && (!w_a || !w2_a)) || (n_b && (!w_b || !w2_b))) return RFR_E_INVALID;
    if (((uintptr_t)workspace) & 255) return RFR_E_INVALID;
    if (n_b <= SMALL_MAX_H && fuse != FUSE_ALWAYS) {
        if (window >= (1ull << 62)) return RFR_E_WINDOW;
        SmallJob sj;
        sj.w_a = w_a; sj.w2_a = w2_a; sj.w_b = w_b; sj.w2_b = w2_b;
        sj.n_a = n_a; sj.n_b = n_b; sj.W = window; sj.W2 = window2;
        sj.cand = cand; sj.cap = cap; sj.ctr = (unsigned long long*)counters;
        cudaStream_t s = (cudaStream_t)stream;
        if (cudaMemsetAsync(counters, 0, 6 * sizeof(uint64_t), s) != cudaSuccess) return RFR_E_CUDA;
        return run_small(&sj, 1, (SmallJob*)workspace, s) == cudaSuccess ? RFR_OK : RFR_E_CUDA;
    }
    MatchGeom g;
    if (!stage_geom(n_a, n_b, window, &g, optimistic, fuse)) return RFR_E_WINDOW;
    const size_t need = g.fused ? g.bytes - align256(mitm_hit_cap(g) * 8) + 8 : g.bytes;   // fused: hits may be fewer
    if (need + 2048 > workspace_bytes) return RFR_E_INVALID;
    char* base = (char*)workspace;
    ProbJob* dev_job = (ProbJob*)base;
    HalfJob* dev_halves = (HalfJob*)(base + 1024);
    ProbJob pj;
    memset(&pj, 0, sizeof(pj));
    match_layout(g, base + 2048, &pj);
    if (g.fused) {                         // hits: whatever the workspace holds beyond the lists
        const size_t used = 2048 + (g.bytes - align256(pj.hcap * 8));
        const uint64_t room = workspace_bytes > used ? (uint64_t)((workspace_bytes - used) / 8) : 0;
        if (room < pj.hcap) pj.hcap = room;
    }
    pj.A.err = pj.B.err = (int*)(counters + 4);
    pj.A.w = w_a; pj.B.w = w_b;
    pj.w_a = w_a; pj.w2_a = w2_a; pj.w_b = w_b; pj.w2_b = w2_b;
    pj.W = window; pj.W2 = window2;
    pj.cand = cand; pj.cap = cap;
    pj.ctr = (unsigned long long*)counters;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(counters, 0, 6 * sizeof(uint64_t), s) != cudaSuccess) return RFR_E_CUDA;
    if (!g.fused &&
        cudaMemsetAsync(g.optimistic ? (void*)pj.A.bcount : (void*)pj.B.halo_cnt, 0,
                        (g.optimistic ? 3 * (((((size_t)1 << g.d1) * 4) + 255) & ~(size_t)255)
                                      : (((size_t)1 << g.d1) + 1) * 4), s) != cudaSuccess) return RFR_E_CUDA;
    HalfJob halves[2];
    cudaError_t e = run_match(&pj, 1, dev_job, dev_halves, halves, s, nullptr, nullptr);
    return e == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}

extern "C" int rfr_stage_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                               const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                               uint64_t window, uint64_t window2,
                               void* workspace, size_t workspace_bytes,
                               uint64_t* cand, uint64_t cap, uint64_t* counters, void* stream) {
    return stage_match(w_a, w2_a, n_a, w_b, w2_b, n_b, window, window2, workspace, workspace_bytes,
                       cand, cap, counters, stream, true);
}

extern "C" int rfr_stage_match_exact(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                                     const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                                     uint64_t window, uint64_t window2,
                                     void* workspace, size_t workspace_bytes,
                                     uint64_t* cand, uint64_t cap, uint64_t* counters, void* stream) {
    return stage_match(w_a, w2_a, n_a, w_b, w2_b, n_b, window, window2, workspace, workspace_bytes,
                       cand, cap, counters, stream, false);
}

extern "C" int rfr_stage_match_fused(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                                     const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                                     uint64_t window, uint64_t window2,
                                     void* workspace, size_t workspace_bytes,
                                     uint64_t* cand, uint64_t cap, uint64_t* counters, void* stream) {
    return stage_match(w_a, w2_a, n_a, w_b, w2_b, n_b, window, window2, workspace, workspace_bytes,
                       cand, cap, counters, stream, true, FUSE_ALWAYS);
}
