// hs_mt.cpp — multithreaded CPU Horowitz–Sahni band join: the CPU baseline
// for the match stage, timed beside the GPU path.  It is neither the oracle
// nor part of the product path.
//
// What it computes is the match of Section 3.3 (EXPAND's sums of both halves,
// their sort, FIND) with FIND's acceptance made circular (Eq. 9 in units of
// 2^-64) and every pair in the window reported, plus the Tr_2 prefilter of
// Section 2:
//   pairs within W:  dist((sum_{i in s_a} w_a[i] + sum_{j in s_b} w_b[j]) mod 2^64) <= W
//   candidates:      those also within W2 for the w2 weights, (s_a, s_b) != (0, 0)
// with dist(y) = min(y, 2^64 - y).  A candidate is written as the pattern
// s_a | s_b << n_a.
//
// Two designs, both on all cores (std::thread):
//
// Runs (halves of at least 12 elements and windows narrow next to a key
// unit), the same design as the GPU's fused match, without a sort of either
// half:
//   lists      each half's h elements split into low elements 0..l-1 and high
//              elements l..h-1; the sorted list Y of all 2^l exact low-subset
//              sums (with masks) is built by merging (the list of i elements
//              merged with its copy shifted by w_i); every high subset x gives
//              one sorted run x + Y (rotated to start at its smallest key);
//   units      the key space is cut into units of about 2^15 keys of half a;
//              threads take ranges of consecutive units and keep a cursor per
//              run; per unit, half a's keys are counting-sorted into 2^14
//              bins in cache and mark an occupancy bitmap, and every key of
//              half b within W of the unit whose bitmap cell is marked looks
//              at the bins its window covers.
// Sorted (small halves, or wide windows):
//   enumerate  key[s] = lo[s & (2^L - 1)] + hi[s >> L] from two half tables,
//              keys of half b negated, so a pair matches when key_a - key_b
//              is within W of 0 mod 2^64;
//   sort       parallel LSD radix sort of (key, mask) on 11-bit digits, one
//              histogram per thread and digit, passes with one occupied
//              digit skipped;
//   join       sorted half a cut into chunks taken dynamically by the
//              threads; each chunk walks half b with one monotone pointer
//              (binary search for the two pieces of a window that wraps).
// Buffers are kept between calls (the function is not reentrant).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <cstdint>
#include <memory>
#include <thread>
#include <vector>

namespace {

template <class F>
void parallel_for(int T, F f) {
    std::vector<std::thread> th;
    th.reserve(T > 1 ? T - 1 : 0);
    for (int t = 1; t < T; ++t) th.emplace_back(f, t);
    f(0);
    for (auto& x : th) x.join();
}

inline size_t part(size_t n, int t, int T) { return n * (size_t)t / (size_t)T; }

// Keys and masks of one half with their radix-sort ping-pong copies.  The
// arrays are left uninitialised on allocation, so their pages are first
// touched by the parallel enumeration and sort.
struct Half {
    std::unique_ptr<uint64_t[]> key, key2;
    std::unique_ptr<uint32_t[]> mask, mask2;
    size_t cap = 0;
    std::vector<uint64_t> t2lo, t2hi;     // Tr_2 sums: t2lo[s & low] + t2hi[s >> L]
    int L = 0;
};

Half g_a, g_b;

void subset_sums(const uint64_t* w, int k, bool neg, std::vector<uint64_t>& t) {
    t.assign((size_t)1 << k, 0);
    for (int i = 0; i < k; ++i) {
        uint64_t wi = neg ? (uint64_t)0 - w[i] : w[i];
        size_t half = (size_t)1 << i;
        for (size_t m = 0; m < half; ++m) t[m | half] = t[m] + wi;
    }
}

void enumerate(const uint64_t* w, const uint64_t* w2, int h, bool neg, int T, Half& H) {
    size_t N = (size_t)1 << h;
    int L = h / 2;
    H.L = L;
    std::vector<uint64_t> lo, hi;
    subset_sums(w, L, neg, lo);
    subset_sums(w + L, h - L, neg, hi);
    subset_sums(w2, L, false, H.t2lo);
    subset_sums(w2 + L, h - L, false, H.t2hi);
    if (H.cap < N) {
        H.key.reset(new uint64_t[N]);  H.key2.reset(new uint64_t[N]);
        H.mask.reset(new uint32_t[N]); H.mask2.reset(new uint32_t[N]);
        H.cap = N;
    }
    size_t lm = ((size_t)1 << L) - 1;
    parallel_for(T, [&](int t) {
        for (size_t m = part(N, t, T), e = part(N, t + 1, T); m < e; ++m) {
            H.key[m] = lo[m & lm] + hi[m >> L];
            H.mask[m] = (uint32_t)m;
        }
    });
}

void radix_sort(size_t N, int T, Half& H) {
    constexpr int DB = 11, NBK = 1 << DB;
    std::vector<size_t> hist((size_t)T * NBK);
    uint64_t* k = H.key.get();  uint64_t* k2 = H.key2.get();
    uint32_t* m = H.mask.get(); uint32_t* m2 = H.mask2.get();
    for (int sh = 0; sh < 64; sh += DB) {
        std::fill(hist.begin(), hist.end(), 0);
        parallel_for(T, [&](int t) {
            size_t* h = &hist[(size_t)t * NBK];
            for (size_t i = part(N, t, T), e = part(N, t + 1, T); i < e; ++i) h[(k[i] >> sh) & (NBK - 1)]++;
        });
        bool trivial = false;
        size_t run = 0;
        for (int d = 0; d < NBK; ++d) {
            size_t tot = 0;
            for (int t = 0; t < T; ++t) tot += hist[(size_t)t * NBK + d];
            if (tot == N) trivial = true;
        }
        if (trivial) continue;
        for (int d = 0; d < NBK; ++d)
            for (int t = 0; t < T; ++t) {
                size_t c = hist[(size_t)t * NBK + d];
                hist[(size_t)t * NBK + d] = run;
                run += c;
            }
        parallel_for(T, [&](int t) {
            size_t* o = &hist[(size_t)t * NBK];
            for (size_t i = part(N, t, T), e = part(N, t + 1, T); i < e; ++i) {
                size_t p = o[(k[i] >> sh) & (NBK - 1)]++;
                k2[p] = k[i];
                m2[p] = m[i];
            }
        });
        std::swap(k, k2);
        std::swap(m, m2);
    }
    if (k != H.key.get()) { H.key.swap(H.key2); H.mask.swap(H.mask2); }
}

inline uint64_t circ(uint64_t y) { return y < (uint64_t)0 - y ? y : (uint64_t)0 - y; }

// ---- runs design
struct RunHalf {
    int h = 0, l = 0;
    uint32_t N = 1, R = 1;              // list entries, runs
    std::vector<uint64_t> Y;            // sorted exact low-subset sums (negated for half b)
    std::vector<uint32_t> M;            // their masks
    std::vector<uint64_t> x;            // run offsets (high-subset sums)
    std::vector<uint32_t> j0;           // index of each run's smallest key
    uint64_t key(uint32_t g, uint64_t t) const { return x[g] + Y[(j0[g] + t) & (N - 1)]; }
    uint32_t mask(uint32_t g, uint64_t t) const { return (g << l) | M[(j0[g] + t) & (N - 1)]; }
    // first rotated index t in [0, N] of run g with key >= v
    uint64_t lower(uint32_t g, uint64_t v) const {
        uint64_t lo = 0, hi = N;
        while (lo < hi) {
            const uint64_t mid = (lo + hi) >> 1;
            if (key(g, mid) < v) lo = mid + 1; else hi = mid;
        }
        return lo;
    }
};

RunHalf g_ra, g_rb;

// Y by merging: the sorted sums of elements 0..i-1 and their copy shifted by
// w_i, which is sorted once rotated to the first entry that wraps past 2^64.
void build_runs(const uint64_t* w, int h, bool neg, RunHalf& H) {
    H.h = h;
    H.l = h <= 7 ? 0 : h - 7;
    H.N = 1u << H.l;
    H.R = 1u << (h - H.l);
    std::vector<uint64_t> K(1, 0), K2;
    std::vector<uint32_t> Mk(1, 0), M2;
    for (int i = 0; i < H.l; ++i) {
        const uint64_t c = neg ? (uint64_t)0 - w[i] : w[i];
        const size_t n = K.size();
        const size_t r = std::lower_bound(K.begin(), K.end(), (uint64_t)0 - c) - K.begin();
        K2.resize(2 * n);
        M2.resize(2 * n);
        size_t a = 0, b = 0, d = 0;
        const size_t nm = n - 1;                                  // n is a power of two
        auto bk = [&](size_t t) { return K[(r + t) & nm] + c; };
        while (a < n || b < n) {
            if (b >= n || (a < n && K[a] <= bk(b))) { K2[d] = K[a]; M2[d++] = Mk[a++]; }
            else { K2[d] = bk(b); M2[d++] = Mk[(r + b) & nm] | (1u << i); ++b; }
        }
        K.swap(K2);
        Mk.swap(M2);
    }
    H.Y.swap(K);
    H.M.swap(Mk);
    H.x.assign(H.R, 0);
    H.j0.assign(H.R, 0);
    for (uint32_t g = 0; g < H.R; ++g) {
        uint64_t s = 0;
        for (int k = 0; k < h - H.l; ++k)
            if ((g >> k) & 1) s += neg ? (uint64_t)0 - w[H.l + k] : w[H.l + k];
        H.x[g] = s;
        H.j0[g] = (uint32_t)((std::lower_bound(H.Y.begin(), H.Y.end(), (uint64_t)0 - s) - H.Y.begin()) & (H.N - 1));
    }
}

// Every pair of keys within W, unit by unit (see the file header).
template <class Emit>
void join_runs(const RunHalf& A, const RunHalf& B, uint64_t W, int T, Emit emit_pair) {
    const int d1 = A.h > 15 ? A.h - 15 : 0;
    const uint64_t NU = 1ull << d1;
    const int su = 64 - d1;
    const int BL = 14, bs = su - BL;                        // 2^14 bins per unit
    // occupancy bitmap of about 2^19 cells per unit: a key of half b is looked
    // up only when its cell holds a key of half a's windows (used when a
    // window spans at most three cells)
    const int cs = su - 19;
    const bool use_bm = ((2 * W) >> cs) <= 2;
    const size_t bm_words = ((((uint64_t)1 << 19) + 8) >> 6) + 2;
    const uint64_t UM = d1 ? (~0ull >> d1) : ~0ull;          // unit width - 1
    const uint64_t per = NU >= (uint64_t)T * 16 ? NU / ((uint64_t)T * 16) : 1;
    std::atomic<uint64_t> next{0};
    parallel_for(T, [&](int) {
        std::vector<uint64_t> ka, sa;
        std::vector<uint32_t> ma, sm, cnt(((size_t)1 << BL) + 1);      // + one bin for the shift by W
        ka.reserve((size_t)1 << 16); ma.reserve((size_t)1 << 16);
        std::vector<uint64_t> bm(bm_words);
        std::vector<uint64_t> ca(A.R), cb(B.R);
        for (;;) {
            const uint64_t u0 = next.fetch_add(per);
            if (u0 >= NU) break;
            const uint64_t u1 = std::min(NU, u0 + per);
            for (uint32_t g = 0; g < A.R; ++g) ca[g] = u0 ? A.lower(g, u0 << su) : 0;
            for (uint32_t g = 0; g < B.R; ++g) cb[g] = u0 ? B.lower(g, (u0 << su) - W) : 0;
            for (uint64_t u = u0; u < u1; ++u) {
                const uint64_t lo = d1 ? u << su : 0;
                const bool last = u == NU - 1;
                // half a: keys in [lo, lo + U), relative to lo, counting-sorted into bins
                ka.clear(); ma.clear();
                for (uint32_t g = 0; g < A.R; ++g) {
                    uint64_t t = ca[g];
                    for (; t < A.N; ++t) {
                        const uint64_t rel = A.key(g, t) - lo;
                        if (!last && rel > UM) break;
                        ka.push_back(rel);
                        ma.push_back(A.mask(g, t));
                    }
                    ca[g] = t;
                }
                // bins over q = key - lo + W (>= 0 for every key within W of the unit)
                std::fill(cnt.begin(), cnt.end(), 0u);
                for (uint64_t& r : ka) { r += W; cnt[r >> bs]++; }
                if (use_bm) {
                    std::fill(bm.begin(), bm.end(), 0ull);
                    for (uint64_t r : ka)
                        for (uint64_t c = (r - W) >> cs, ce = (r + W) >> cs; c <= ce; ++c) bm[c >> 6] |= 1ull << (c & 63);
                }
                uint32_t run = 0;
                for (auto& c : cnt) { const uint32_t v = c; c = run; run += v; }
                sa.resize(ka.size()); sm.resize(ka.size());
                for (size_t i = 0; i < ka.size(); ++i) {
                    const uint32_t p = cnt[ka[i] >> bs]++;
                    sa[p] = ka[i]; sm[p] = ma[i];
                }
                // now cnt[k] = end of bin k
                const uint32_t* cn = cnt.data();
                const uint64_t* sp = sa.data();
                const uint32_t* smp = sm.data();
                const uint64_t kmax = cnt.size() - 1;
                auto probe = [&](uint64_t kb, uint32_t mb) {
                    const uint64_t q = kb - lo + W;                     // in [0, U + 2 W)
                    if (use_bm) {
                        const uint64_t c = q >> cs;
                        if (!((bm[std::min<uint64_t>(c >> 6, bm_words - 1)] >> (c & 63)) & 1)) return;
                    }
                    const uint64_t blo = q < W ? 0 : (q - W) >> bs;
                    const uint64_t bhi = std::min(kmax, (q + W) >> bs);
                    for (uint64_t k = blo; k <= bhi; ++k)
                        for (uint32_t i = k ? cn[k - 1] : 0; i < cn[k]; ++i)
                            if (circ(sp[i] - q) <= W) emit_pair(smp[i], mb);
                };
                // half b: keys in [lo - W, lo + U + W) (circularly)
                for (uint32_t g = 0; g < B.R; ++g) {
                    uint64_t t = cb[g];
                    for (; t < B.N; ++t) {
                        const uint64_t kb = B.key(g, t);
                        if (!last && kb - lo + W > UM + 2 * W) break;     // beyond lo + U + W
                        probe(kb, B.mask(g, t));
                    }
                    // next unit's first key: the first >= lo + U - W
                    uint64_t nt = cb[g];
                    if (!last) while (nt < B.N && B.key(g, nt) - lo + W < UM + 1) ++nt;
                    cb[g] = nt;
                    if (u == 0)                               // keys in [2^64 - W, 2^64) meet unit 0
                        for (uint64_t s = B.lower(g, (uint64_t)0 - W); W && s < B.N && B.key(g, s) >= (uint64_t)0 - W; ++s)
                            probe(B.key(g, s), B.mask(g, s));
                    if (last && NU > 1)                       // keys in [0, W) meet the last unit
                        for (uint64_t s = 0; s < B.N && B.key(g, s) < W; ++s) probe(B.key(g, s), B.mask(g, s));
                }
            }
        }
    });
}

}  // namespace

extern "C" {

// Returns 0, or -1 on invalid arguments.  counts[3] receives {pairs within W
// (the trivial pair included), candidates, trivial pair seen}; at most cap
// candidates are written to pairs (counts[1] is the full count).
// seconds[3] (if given) receives the enumerate (the runs design: list build),
// sort (runs: 0) and join times.
int hs_mt_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                uint64_t W, uint64_t W2, int threads,
                uint64_t* pairs, uint64_t cap, uint64_t* counts, double* seconds) {
    if (n_a < 0 || n_b < 0 || n_a + n_b > 63 || n_a > 32 || n_b > 32 || !counts) return -1;
    if (W >= ((uint64_t)1 << 63)) return -1;
    int T = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto t0 = now();
    // runs design: halves of at least 16 elements (two key units or more) and a
    // window narrower than a sixteenth of a unit
    if (n_a >= 16 && n_b >= n_a && W < ((uint64_t)1 << (64 - (n_a - 15) - 4))) {
        std::thread tb([&] { build_runs(w_b, n_b, true, g_rb); });
        build_runs(w_a, n_a, false, g_ra);
        tb.join();
        const int La = n_a / 2, Lb = n_b / 2;
        std::vector<uint64_t> t2la, t2ha, t2lb, t2hb;
        subset_sums(w2_a, La, false, t2la); subset_sums(w2_a + La, n_a - La, false, t2ha);
        subset_sums(w2_b, Lb, false, t2lb); subset_sums(w2_b + Lb, n_b - Lb, false, t2hb);
        const uint32_t lma = (1u << La) - 1, lmb = (1u << Lb) - 1;
        auto t1 = now();
        std::atomic<uint64_t> within{0}, cands{0}, trivial{0};
        join_runs(g_ra, g_rb, W, T, [&](uint32_t sa, uint32_t sb) {
            within.fetch_add(1, std::memory_order_relaxed);
            if (sa == 0 && sb == 0) { trivial.store(1); return; }
            const uint64_t t2 = t2la[sa & lma] + t2ha[sa >> La] + t2lb[sb & lmb] + t2hb[sb >> Lb];
            if (circ(t2) > W2) return;
            const uint64_t p = cands.fetch_add(1);
            if (p < cap && pairs) pairs[p] = (uint64_t)sa | ((uint64_t)sb << n_a);
        });
        auto t2 = now();
        counts[0] = within.load();
        counts[1] = cands.load();
        counts[2] = trivial.load();
        if (seconds) {
            seconds[0] = std::chrono::duration<double>(t1 - t0).count();
            seconds[1] = 0.0;
            seconds[2] = std::chrono::duration<double>(t2 - t1).count();
        }
        return 0;
    }
    enumerate(w_a, w2_a, n_a, false, T, g_a);
    enumerate(w_b, w2_b, n_b, true, T, g_b);
    auto t1 = now();
    size_t NA = (size_t)1 << n_a, NB = (size_t)1 << n_b;
    radix_sort(NA, T, g_a);
    radix_sort(NB, T, g_b);
    auto t2 = now();
    const uint64_t* A = g_a.key.get();  const uint32_t* MA = g_a.mask.get();
    const uint64_t* B = g_b.key.get();  const uint32_t* MB = g_b.mask.get();
    const size_t lma = ((size_t)1 << g_a.L) - 1, lmb = ((size_t)1 << g_b.L) - 1;
    std::atomic<uint64_t> within{0}, cands{0}, trivial{0};
    std::atomic<size_t> next{0};
    size_t chunk = std::max<size_t>(1024, NA / ((size_t)T * 64));
    parallel_for(T, [&](int) {
        uint64_t my_w = 0;
        auto emit = [&](size_t i, size_t k) {
            ++my_w;
            uint32_t sa = MA[i], sb = MB[k];
            if (sa == 0 && sb == 0) { trivial.store(1); return; }
            uint64_t t2 = g_a.t2lo[sa & lma] + g_a.t2hi[sa >> g_a.L] + g_b.t2lo[sb & lmb] + g_b.t2hi[sb >> g_b.L];
            if (circ(t2) > W2) return;
            uint64_t p = cands.fetch_add(1);
            if (p < cap && pairs) pairs[p] = (uint64_t)sa | ((uint64_t)sb << n_a);
        };
        for (;;) {
            size_t b = next.fetch_add(chunk);
            if (b >= NA) break;
            size_t e = std::min(NA, b + chunk);
            uint64_t a0 = A[b];
            size_t lo = a0 >= W ? std::lower_bound(B, B + NB, a0 - W) - B : 0;
            for (size_t i = b; i < e; ++i) {
                uint64_t a = A[i], x = a - W, y = a + W;
                if (a >= W && a <= ~(uint64_t)0 - W) {
                    while (lo < NB && B[lo] < x) ++lo;
                    for (size_t k = lo; k < NB && B[k] <= y; ++k) emit(i, k);
                } else {                         // the window wraps: [x, 2^64) and [0, y]
                    for (size_t k = std::lower_bound(B, B + NB, x) - B; k < NB; ++k) emit(i, k);
                    for (size_t k = 0; k < NB && B[k] <= y; ++k) emit(i, k);
                }
            }
        }
        within.fetch_add(my_w);
    });
    auto t3 = now();
    counts[0] = within.load();
    counts[1] = cands.load();
    counts[2] = trivial.load();
    if (seconds) {
        seconds[0] = std::chrono::duration<double>(t1 - t0).count();
        seconds[1] = std::chrono::duration<double>(t2 - t1).count();
        seconds[2] = std::chrono::duration<double>(t3 - t2).count();
    }
    return 0;
}

}  // extern "C"
