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
//  * K-c + radix digit 1 (top d1 key bits, 4..8192 buckets):
//      k_count   — Gray-code enumeration of every pattern, per-CTA bucket
//                  histogram in shared memory;
//      k_colscan / k_bscan — per-CTA offsets and bucket starts;
//      k_scatter — the same enumeration again, each record written to its
//                  bucket at a shared-memory cursor, so every CTA fills a
//                  contiguous run of each bucket.
//    Record (8 bytes): ((key << d1) & ~(2^h - 1)) | mask.  The top d1 key
//    bits are implied by the bucket, so the record keeps key bits
//    [63-d1 .. h-d1] and the pattern's mask; the truncation is below
//    2^max(0, h-d1).
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

// ---------------------------------------------------------------- K-c + digit 1
__global__ void __launch_bounds__(PART_THREADS) k_count(const HalfJob* __restrict__ hs, int nh) {
    extern __shared__ uint32_t sh_hist[];
    __shared__ uint64_t sw[32];
    const int j = find_last_le(nh, (int)blockIdx.x, [&](int i) { return hs[i].cta_base; });
    const HalfJob J = hs[j];
    const int c = blockIdx.x - J.cta_base;
    const int d1 = J.d1, NB = 1 << d1, sh = 64 - d1;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) sh_hist[b] = 0u;
    if (threadIdx.x < J.h) sw[threadIdx.x] = J.w[threadIdx.x];
    __syncthreads();
    const uint64_t per = (1ull << J.h) / (uint64_t)J.ctas;
    const int tr = J.h > d1 ? J.h - d1 : 0;
    const uint64_t trunc = lowmask(tr);
    const uint64_t width = 1ull << sh, wc = J.wc;
    const int neg = J.neg;
    uint32_t* halo_cnt = J.halo_cnt;
    enumerate_range(sw, per * (uint64_t)c, per, [&](uint64_t m, uint64_t key) {
        const uint64_t K = neg ? (0ull - key) : key;
        const uint32_t b = (uint32_t)(K >> sh);
        atomicAdd(&sh_hist[b], 1u);
        if (neg) {
            const uint64_t off = (K & ~trunc) - ((uint64_t)b << sh);
            if (off < wc) atomicAdd(&halo_cnt[(b - 1u) & (uint32_t)(NB - 1)], 1u);
            if (width - off <= wc) atomicAdd(&halo_cnt[(b + 1u) & (uint32_t)(NB - 1)], 1u);
        }
    });
    __syncthreads();
    uint32_t* out = J.hist + (size_t)c * NB;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) out[b] = sh_hist[b];
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

__global__ void __launch_bounds__(PART_THREADS) k_scatter(const HalfJob* __restrict__ hs, int nh) {
    extern __shared__ uint32_t cur[];
    __shared__ uint64_t sw[32];
    const int j = find_last_le(nh, (int)blockIdx.x, [&](int i) { return hs[i].cta_base; });
    const HalfJob J = hs[j];
    const int c = blockIdx.x - J.cta_base;
    const int d1 = J.d1, NB = 1 << d1, sh = 64 - d1;
    for (int b = threadIdx.x; b < NB; b += blockDim.x) cur[b] = J.bstart[b] + J.hist[(size_t)c * NB + b];
    if (threadIdx.x < J.h) sw[threadIdx.x] = J.w[threadIdx.x];
    __syncthreads();
    const uint64_t per = (1ull << J.h) / (uint64_t)J.ctas;
    const uint64_t lm = lowmask(J.h);
    const int tr = J.h > d1 ? J.h - d1 : 0;
    const uint64_t trunc = lowmask(tr);
    const uint64_t width = 1ull << sh, wc = J.wc, hcap = J.halo_cap;
    const int neg = J.neg;
    uint64_t* tab = J.tab;
    uint64_t* halo = J.halo;
    uint32_t* halo_cur = J.halo_cur;
    enumerate_range(sw, per * (uint64_t)c, per, [&](uint64_t m, uint64_t key) {
        const uint64_t K = neg ? (0ull - key) : key;
        const uint32_t b = (uint32_t)(K >> sh);
        const uint32_t p = atomicAdd(&cur[b], 1u);
        tab[p] = ((K << d1) & ~lm) | m;
        if (neg) {
            const uint64_t Kc = K & ~trunc;
            const uint64_t off = Kc - ((uint64_t)b << sh);
            if (off < wc) {
                const uint32_t hp = atomicAdd(&halo_cur[(b - 1u) & (uint32_t)(NB - 1)], 1u);
                if (hp < hcap) { halo[2 * (size_t)hp] = Kc; halo[2 * (size_t)hp + 1] = m; }
            }
            if (width - off <= wc) {
                const uint32_t hp = atomicAdd(&halo_cur[(b + 1u) & (uint32_t)(NB - 1)], 1u);
                if (hp < hcap) { halo[2 * (size_t)hp] = Kc; halo[2 * (size_t)hp + 1] = m; }
            }
        }
    });
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
    const uint32_t a0 = P.A.bstart[k], a1 = P.A.bstart[k + 1];
    const uint32_t b0 = P.B.bstart[k], b1 = P.B.bstart[k + 1];
    const uint64_t hcap = P.B.halo_cap;
    const uint32_t h0 = (uint32_t)min((uint64_t)P.B.halo_cnt[k], hcap);
    const uint32_t h1 = (uint32_t)min((uint64_t)P.B.halo_cnt[k + 1], hcap);
    const uint32_t nbn = b1 - b0, nbt = nbn + (h1 - h0);
    const uint64_t Wc = P.Wc, W = P.W, W2 = P.W2;
    const uint64_t* __restrict__ tabA = P.A.tab;
    const uint64_t* __restrict__ tabB = P.B.tab;
    const uint64_t* __restrict__ halo = P.B.halo;
    unsigned long long n_coarse = 0, n_pre = 0;
    __syncthreads();
    for (uint32_t cs = a0; cs < a1; cs += JOIN_CAP) {
        const uint32_t m = min((uint32_t)JOIN_CAP, a1 - cs);
        for (int s = threadIdx.x; s < (1 << SUB_BITS); s += blockDim.x) off[s] = 0u;
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
            const uint64_t r = tabA[cs + i];
            const uint64_t dk = (r & ~la) >> d1;          // key offset inside the bucket
            atomicAdd(&off[dk >> subsh], 1u);
        }
        __syncthreads();
        block_scan_array(off, 1 << SUB_BITS, false, warp_sums);
        __syncthreads();
        for (uint32_t i = threadIdx.x; i < m; i += blockDim.x) {
            const uint64_t r = tabA[cs + i];
            const uint64_t dk = (r & ~la) >> d1;
            const uint32_t p = atomicAdd(&off[dk >> subsh], 1u);
            As[p] = r;
        }
        __syncthreads();
        for (uint32_t t = threadIdx.x; t < nbt; t += blockDim.x) {
            uint64_t Kb, mb;
            if (t < nbn) {
                const uint64_t r = tabB[b0 + t];
                Kb = lo_k | ((r & ~lb) >> d1);
                mb = r & lb;
            } else {
                const size_t hi = 2 * (size_t)(h0 + (t - nbn));
                Kb = halo[hi];
                mb = halo[hi + 1];
            }
            long long dlo = (long long)(Kb - Wc + 1ull - lo_k);
            long long dhi = (long long)(Kb + Wc - 1ull - lo_k);
            if (dhi < 0 || dlo >= width) continue;
            if (dlo < 0) dlo = 0;
            if (dhi > width - 1) dhi = width - 1;
            const int s_lo = (int)(dlo >> subsh), s_hi = (int)(dhi >> subsh);
            const uint32_t p0 = s_lo ? off[s_lo - 1] : 0u, p1 = off[s_hi];
            for (uint32_t p = p0; p < p1; ++p) {
                const uint64_t ra = As[p];
                const uint64_t Ka = lo_k | ((ra & ~la) >> d1);
                const long long diff = (long long)(Ka - Kb);
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
        }
        __syncthreads();
    }
    if (n_coarse) atomicAdd(&P.ctr[0], n_coarse);
    if (n_pre) atomicAdd(&P.ctr[1], n_pre);
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
    const size_t NB = (size_t)1 << g.d1;
    size_t b = 0;
    b += align256(((size_t)1 << g.n_a) * 8);
    b += align256(((size_t)1 << g.n_b) * 8);
    b += align256((size_t)g.ctas_a * NB * 4);
    b += align256((size_t)g.ctas_b * NB * 4);
    b += 2 * align256((NB + 1) * 4);
    b += align256((NB + 1) * 4) + align256(NB * 4);
    b += align256((size_t)g.hcap * 16);
    return b;
}

bool match_geometry(int n_a, int n_b, uint64_t W, int ctas_a, int ctas_b, MatchGeom* g) {
    if (n_a < 0 || n_b < n_a || n_b > 32) return false;
    int d1 = n_a - 13;
    if (d1 < 2) d1 = 2;
    if (d1 > MAX_D1) d1 = MAX_D1;
    uint64_t wc = 0;
    for (; d1 >= 2; --d1) {
        const int tr = n_b > d1 ? n_b - d1 : 0;
        wc = W + (1ull << tr);
        if (wc < W) continue;                                  // overflow
        if (wc < (1ull << (64 - d1)) / 4) break;
    }
    if (d1 < 2) return false;
    g->n_a = n_a; g->n_b = n_b; g->d1 = d1; g->wc = wc;
    g->ctas_a = ctas_a; g->ctas_b = ctas_b;
    g->hcap = default_halo_cap(n_b, d1, wc);
    g->bytes = match_bytes(*g);
    return true;
}

void match_layout(const MatchGeom& g, char* ws, ProbJob* pj) {
    const size_t NB = (size_t)1 << g.d1;
    char* p = ws;
    auto take = [&](size_t bytes) { char* q = p; p += align256(bytes); return q; };
    HalfJob& A = pj->A;
    HalfJob& B = pj->B;
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
    A.halo_cnt = nullptr; A.halo_cur = nullptr; A.halo = nullptr; A.halo_cap = 0;
    A.h = g.n_a; B.h = g.n_b;
    A.neg = 0; B.neg = 1;
    A.d1 = B.d1 = g.d1;
    A.ctas = g.ctas_a; B.ctas = g.ctas_b;
    A.wc = B.wc = g.wc;
    pj->n_a = g.n_a; pj->n_b = g.n_b; pj->d1 = g.d1; pj->Wc = g.wc;
}

// Assign grid bases for a set of problems; fills halves[2*np].
struct MatchGrid { int part_ctas, scan_ctas, join_ctas, nb_max; };

static MatchGrid assign_bases(ProbJob* jobs, int np, HalfJob* halves) {
    MatchGrid g{0, 0, 0, 0};
    for (int i = 0; i < np; ++i) {
        ProbJob& P = jobs[i];
        const int NB = 1 << P.d1;
        HalfJob* hh[2] = {&P.A, &P.B};
        for (int t = 0; t < 2; ++t) {
            hh[t]->cta_base = g.part_ctas;
            g.part_ctas += hh[t]->ctas;
            hh[t]->scan_base = g.scan_ctas;
            g.scan_ctas += (NB + 255) / 256;
            halves[2 * i + t] = *hh[t];
        }
        P.join_base = g.join_ctas;
        g.join_ctas += NB;
        if (NB > g.nb_max) g.nb_max = NB;
    }
    return g;
}

static bool g_attr_set = false;
static const size_t JOIN_SMEM = (size_t)JOIN_CAP * 8 + ((size_t)1 << SUB_BITS) * 4;

// Upload jobs (from host memory that stays valid until the copies finish:
// pageable memory is staged before cudaMemcpyAsync returns) and launch.
cudaError_t run_match(ProbJob* jobs, int np, ProbJob* dev_jobs, HalfJob* dev_halves,
                      HalfJob* host_halves, cudaStream_t s, cudaEvent_t ev_mid) {
    if (!g_attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_join, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)JOIN_SMEM);
        if (e != cudaSuccess) return e;
        g_attr_set = true;
    }
    MatchGrid g = assign_bases(jobs, np, host_halves);
    cudaError_t e;
    e = cudaMemcpyAsync(dev_halves, host_halves, sizeof(HalfJob) * 2 * np, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    e = cudaMemcpyAsync(dev_jobs, jobs, sizeof(ProbJob) * np, cudaMemcpyHostToDevice, s);
    if (e != cudaSuccess) return e;
    const size_t psmem = (size_t)g.nb_max * 4;
    k_count<<<g.part_ctas, PART_THREADS, psmem, s>>>(dev_halves, 2 * np);
    k_colscan<<<g.scan_ctas, 256, 0, s>>>(dev_halves, 2 * np);
    k_bscan<<<2 * np, 1024, 0, s>>>(dev_halves, 2 * np);
    k_scatter<<<g.part_ctas, PART_THREADS, psmem, s>>>(dev_halves, 2 * np);
    if (ev_mid) cudaEventRecord(ev_mid, s);
    k_join<<<g.join_ctas, JOIN_THREADS, JOIN_SMEM, s>>>(dev_jobs, np);
    return cudaGetLastError();
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
    int c = h > 16 ? 1 << (h - 16) : 1;
    return c > 256 ? 256 : c;
}

// Stage workspace: job structs, then one problem's buffers with a halo large
// enough for every record of table b (so no window can overflow it).
static bool stage_geom(int n_a, int n_b, uint64_t W, MatchGeom* g) {
    if (!match_geometry(n_a, n_b, W, stage_ctas(n_a), stage_ctas(n_b), g)) return false;
    g->hcap = 1ull << n_b;
    g->bytes = match_bytes(*g);
    return true;
}

extern "C" size_t rfr_stage_match_workspace(int n_a, int n_b) {
    MatchGeom g;
    if (!stage_geom(n_a, n_b, 0, &g)) return 0;
    // the bucket count only shrinks for wider windows; budget for d1 = MAX_D1 histograms
    const size_t hist_extra = ((size_t)stage_ctas(n_a) + stage_ctas(n_b)) * ((size_t)1 << MAX_D1) * 4 + 8 * 4096;
    return g.bytes + hist_extra + 2048;
}

extern "C" int rfr_stage_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                               const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                               uint64_t window, uint64_t window2,
                               void* workspace, size_t workspace_bytes,
                               uint64_t* cand, uint64_t cap, uint64_t* counters, void* stream) {
    if (n_a < 0 || n_b < n_a || n_b > 32 || !workspace || !counters || (!cand && cap)) return RFR_E_INVALID;
    if ((n_a && (!w_a || !w2_a)) || (n_b && (!w_b || !w2_b))) return RFR_E_INVALID;
    if (((uintptr_t)workspace) & 255) return RFR_E_INVALID;
    MatchGeom g;
    if (!stage_geom(n_a, n_b, window, &g)) return RFR_E_WINDOW;
    if (g.bytes + 2048 > workspace_bytes) return RFR_E_INVALID;
    char* base = (char*)workspace;
    ProbJob* dev_job = (ProbJob*)base;
    HalfJob* dev_halves = (HalfJob*)(base + 1024);
    ProbJob pj;
    memset(&pj, 0, sizeof(pj));
    match_layout(g, base + 2048, &pj);
    pj.A.err = pj.B.err = (int*)(counters + 4);
    pj.A.w = w_a; pj.B.w = w_b;
    pj.w_a = w_a; pj.w2_a = w2_a; pj.w_b = w_b; pj.w2_b = w2_b;
    pj.W = window; pj.W2 = window2;
    pj.cand = cand; pj.cap = cap;
    pj.ctr = (unsigned long long*)counters;
    cudaStream_t s = (cudaStream_t)stream;
    if (cudaMemsetAsync(counters, 0, 6 * sizeof(uint64_t), s) != cudaSuccess) return RFR_E_CUDA;
    if (cudaMemsetAsync(pj.B.halo_cnt, 0, (((size_t)1 << g.d1) + 1) * 4, s) != cudaSuccess) return RFR_E_CUDA;
    HalfJob halves[2];
    cudaError_t e = run_match(&pj, 1, dev_job, dev_halves, halves, s, nullptr);
    return e == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
