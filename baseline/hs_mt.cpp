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
// Design (a plain CPU Horowitz–Sahni on all cores, std::thread):
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

}  // namespace

extern "C" {

// Returns 0, or -1 on invalid arguments.  counts[3] receives {pairs within W
// (the trivial pair included), candidates, trivial pair seen}; at most cap
// candidates are written to pairs (counts[1] is the full count).
// seconds[3] (if given) receives the enumerate, sort and join times.
int hs_mt_match(const uint64_t* w_a, const uint64_t* w2_a, int n_a,
                const uint64_t* w_b, const uint64_t* w2_b, int n_b,
                uint64_t W, uint64_t W2, int threads,
                uint64_t* pairs, uint64_t cap, uint64_t* counts, double* seconds) {
    if (n_a < 0 || n_b < 0 || n_a + n_b > 63 || n_a > 32 || n_b > 32 || !counts) return -1;
    if (W >= ((uint64_t)1 << 63)) return -1;
    int T = threads > 0 ? threads : (int)std::max(1u, std::thread::hardware_concurrency());
    auto now = [] { return std::chrono::steady_clock::now(); };
    auto t0 = now();
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
