// k_match.cuh — job descriptors shared by the enumerate / partition / match
// kernels (K-c, K-d, K-e) and their host-side planners.
#pragma once
#include <cstdint>
#include <mutex>
#include <vector>
#include <cuda_runtime.h>

namespace rfr {

// A kernel attribute set with cudaFuncSetAttribute holds for the current
// device only: run `set` once per device ordinal (thread-safe), so that a
// process that drives several GPUs sets it on each.
struct PerDeviceOnce {
    static constexpr int kMaxDevices = 64;
    std::mutex mu;
    bool done[kMaxDevices] = {};
    template <class F>
    cudaError_t run(F set) {
        int dev = 0;
        cudaError_t e = cudaGetDevice(&dev);
        if (e != cudaSuccess) return e;
        if (dev < 0 || dev >= kMaxDevices) return cudaErrorInvalidDevice;
        std::lock_guard<std::mutex> lk(mu);
        if (done[dev]) return cudaSuccess;
        e = set();
        if (e == cudaSuccess) done[dev] = true;
        return e;
    }
};

constexpr int SUB_BITS = 13;          // second radix digit, sorted in shared memory
constexpr int JOIN_CAP = 9216;        // table-a entries per shared-memory chunk
constexpr int JOIN_THREADS = 512;
constexpr int PART_THREADS = 512;
constexpr int MAX_D1 = 18;            // first radix digit, at most 262144 buckets
constexpr int YSORT_THREADS = 1024;

// One half-table (a: keys = sum w; b: keys = -sum w) of one problem.
// The half's h elements are split into low bits 0..l-1 (list Y: all 2^l
// low-subset sums, sorted) and high bits l..h-1 (2^hx high subsets x, one
// rotated run x + Y each).
struct HalfJob {
    const uint64_t* w;      // h weights (device)
    int h;                  // elements of this half (mask bits), 0..32
    int neg;                // 1 for half b
    int d1;                 // bucket bits (>= 2)
    int l;                  // low bits (Y list size 2^l)
    int ctas;               // CTAs of the count/scatter grids for this half (<= pieces of 4096)
    int cta_base;           // first CTA of this half in those grids
    int scan_base;          // first CTA of this half in the column-scan grid
    uint64_t wc;            // coarse window (halo test, half b)
    uint64_t* ylist;        // [2^l] sorted (low-subset sum with low l bits cleared) | low mask
    uint64_t* ytmp;         // [2^l] radix-sort ping-pong buffer
    uint32_t* hist;         // [ctas][NB]: counts, then per-CTA offsets
    uint32_t* bstart;       // [NB + 1]: bucket starts in tab
    uint64_t* tab;          // [2^h] records ((key << d1) & ~lowmask) | mask
    uint32_t* halo_cnt;     // [NB + 1] (half b): halo counts, then starts
    uint32_t* halo_cur;     // [NB]     (half b): halo write cursors
    uint64_t* halo;         // [halo_cap][2] (half b): (coarse key, mask)
    uint64_t halo_cap;
    int* err;               // set to 1 on halo or bucket overflow
    // optimistic layout (no count pass): bucket k owns tab[k*opt_cap ..) and
    // halo[k*opt_hcap ..); bcount / hcount are the final cursors (= counts)
    uint32_t opt_cap;       // 0: exact layout from the count pass
    uint32_t opt_hcap;
    uint32_t* bcount;       // [NB]
    uint32_t* hcount;       // [NB] (half b)
    // fused match (k_mitm): ylist holds the exact low-subset sums, ascending;
    // list-building buffers: ytmp is the first key buffer
    uint64_t* kb1;          // [2^(l-1)] second key buffer (l > 13)
    uint32_t* ysplit;       // merge-path tile starts of one level (l > 13)
    uint32_t* ymask;        // [2^l] low-subset mask of each list entry
    uint32_t* ydir;         // [2^l + 1] directory: first entry >= q * 2^(64-l)
    uint32_t* ymtmp[2];     // [2^(l-1)] mask buffers of the levels (l > 13)
    uint32_t* y32;          // [2^l] fused match: bits fsh .. fsh+31 of each list entry
};

// One problem's match.
struct ProbJob {
    HalfJob A, B;
    const uint64_t* w_a;  const uint64_t* w2_a;
    const uint64_t* w_b;  const uint64_t* w2_b;
    int n_a, n_b, d1;
    int join_base;          // first CTA of this problem in the join grid (one per bucket)
    uint64_t W, W2, Wc;
    uint64_t* cand;
    uint64_t cap;
    unsigned long long* ctr;    // [4]: coarse pairs, pairs within W, candidates (within W and W2, non-trivial), trivial seen
    int fused;              // 1: matched by k_mitm (no tables)
    int nbl, slab, wf;      // k_mitm: bins per unit (log2), units per CTA, fingerprint window
    uint64_t* hits;         // k_mitm: fingerprint hits awaiting the exact check (count in ctr[5])
    uint64_t hcap;
    int splat;              // 1: matched by splat sort + query (Algorithm E; ctr has 8 words)
    uint64_t* gamma;        // splat array of half b
    int prune;              // 1: searched by Algorithm B over all n_a + n_b elements
    int shard, nshards;     // fused match: only key-range shard `shard` of `nshards` (0 = all)
};

// One small problem (n_b <= SMALL_MAX_H) matched entirely in shared memory.
constexpr int SMALL_MAX_H = 13;
constexpr int SMALL_THREADS = 512;
struct SmallJob {
    const uint64_t* w_a;  const uint64_t* w2_a;
    const uint64_t* w_b;  const uint64_t* w2_b;
    int n_a, n_b;
    uint64_t W, W2;
    uint64_t* cand;
    uint64_t cap;
    unsigned long long* ctr;    // [6], as ProbJob
};
cudaError_t run_small(const SmallJob* jobs, int np, SmallJob* dev_jobs, cudaStream_t s);
// run_small in two parts: the kernel attribute (once per device), and the
// launch for records already at dev_jobs (no allocation or synchronisation,
// so it may run under stream capture).
cudaError_t small_attrs();
cudaError_t small_issue(const SmallJob* dev_jobs, int np, cudaStream_t s);

// Host-side sizing of one problem's match.
struct MatchGeom {
    int n_a, n_b, d1, ctas_a, ctas_b, l_a, l_b;
    bool optimistic;        // per-bucket slack regions instead of a count pass
    uint32_t cap_a, cap_b;  // optimistic bucket capacities (records)
    uint32_t hcap_per;      // optimistic halo slots per bucket
    uint64_t wc;
    uint64_t hcap;          // halo capacity (entries)
    size_t bytes;           // device workspace bytes (tables + histograms + halo)
    bool fused;             // k_mitm: sorted lists only, units of 2^(64-d1) keys
    int nbl, slab, wf;
    bool splat;             // splat sort + query: one array of 2^(n_b+1) + SPLAT_TAIL cells
    bool prune;             // Algorithm B: no tables at all
};

// Layout knobs chosen by the autotuner.  Table match (defaults 16, 13, 16):
// low-list bits, bucket digit, scatter CTAs per SM.  Fused match (defaults
// 14, 13): the key-unit size, i.e. the mean number of half-a keys a CTA
// holds in its shared-memory table at a time (2^unit_log), and the most bins
// per unit (2^nbl_max).
struct TuneParams {
    int l_max = 16;          // low-list bits (sorted list Y of up to 2^l_max sums)
    int d1_off = 13;         // bucket bits d1 = n_a - d1_off (mean table-a bucket 2^d1_off)
    int cta_per_sm = 16;     // scatter CTAs per SM over a sub-batch
    int unit_log = 14;       // fused: units of 2^unit_log half-a keys on average (12 .. 14)
    int nbl_max = 13;        // fused: at most 2^nbl_max bins per unit (10 .. 13)
};

// Which match a problem gets: tables in device memory, or the fused match
// (k_mitm) for halves of at least FUSED_MIN_NA elements, or only the fused one.
// FUSE_SPLAT: the splat match (Algorithm E) for every problem it fits;
// FUSE_PRUNE: Algorithm B for every problem of at most PRUNE_RUNTIME_MAX_M
// searched elements; other problems get the automatic choice.
enum { FUSE_NEVER = 0, FUSE_AUTO = 1, FUSE_ALWAYS = 2, FUSE_SPLAT = 3, FUSE_PRUNE = 4 };
constexpr int FUSED_MIN_NA = 14;

// Splat match (k_splat.cu): overflow cells past the 2^(n_b+1) home cells.
constexpr uint64_t SPLAT_TAIL = 4096;
bool splat_geometry(int n_a, int n_b, MatchGeom* g);
uint64_t* splat_layout(const MatchGeom& g, char* ws, ProbJob* pj);
// Fill the splat arrays and launch insert + query for S[0..nS); dev_jobs holds
// nS ProbJob slots of device memory.  Two kernel launches.
cudaError_t run_splat(const ProbJob* const* S, int nS, void* dev_jobs, cudaStream_t s);

// Algorithm B (k_prune.cu): at most PRUNE_MAX_M searched elements per stage
// call, PRUNE_RUNTIME_MAX_M in the runtime (its work grows as 2^m / (2^l / l)).
constexpr int PRUNE_MAX_M = 44;
constexpr int PRUNE_RUNTIME_MAX_M = 40;
bool prune_geometry(int n_a, int n_b, MatchGeom* g);
// One kernel launch for P[0..nP); dev_jobs holds nP ProbJob slots.
cudaError_t run_prune(const ProbJob* const* P, int nP, void* dev_jobs, cudaStream_t s);

// Choose bucket bits and coarse window; returns false if the window is too
// wide for any bucket layout.  optimistic = false always gives the table
// match with the exact (count-pass) layout.
bool match_geometry(int n_a, int n_b, uint64_t W, int ctas_a, int ctas_b, MatchGeom* g,
                    bool optimistic = true, const TuneParams* tp = nullptr, int fuse = FUSE_AUTO);

// Geometry of the fused match; false if the halves or the window do not fit it.
// tp (optional) gives the unit size and the bin limit.
bool mitm_geometry(int n_a, int n_b, uint64_t W, MatchGeom* g, const TuneParams* tp = nullptr);
size_t mitm_half_bytes(int l);
uint64_t mitm_hit_cap(const MatchGeom& g);
void mitm_layout_half(int l, char*& p, HalfJob* h);
// Build the sorted lists and run k_mitm for the fused problems F[0..nF);
// dev_mjobs / dev_yjobs hold nF ProbJob / 2*nF HalfJob slots of device memory.
// ev_lists and ev_lists2 (if given) are recorded after the sorted lists are built.
cudaError_t run_mitm(const ProbJob* const* F, int nF, void* dev_mjobs, void* dev_yjobs, cudaStream_t s,
                     cudaEvent_t ev_lists = nullptr, cudaEvent_t ev_lists2 = nullptr);
int mitm_launches(const ProbJob* const* F, int nF);
// run_mitm in two parts, so that the launches can be captured in a CUDA graph
// and replayed with new job records.  mitm_prepare (host only) writes the nF
// MitmJob records (mitm_job_bytes(nF)) to mj_host and the 2 nF list-build
// records (mitm_yjob_bytes(nF)) to yj_host and returns the launch shape;
// mitm_issue launches the list build, k_mitm and k_mitm_check for records
// already at dev_mjobs / dev_yjobs.  mitm_issue allocates nothing, sets no
// attribute and does not synchronise, so it may run under stream capture
// (ev_flags = cudaEventRecordExternal then records the two events in the graph).
struct MitmShape {
    int nF = 0, nh = 0, ctas = 0, dir_lmax = 0;
    int wrap = 0;           // some problem's key positions wrap (k_mitm<true, .>)
    int wide = 0;           // some problem's position lists exceed 32 MB: 16-byte position loads
    std::vector<int> ls;    // list bits of each half in launch order (descending)
};
cudaError_t mitm_prepare(const ProbJob* const* F, int nF, void* mj_host, void* yj_host, MitmShape* sh);
cudaError_t mitm_issue(const MitmShape& sh, void* dev_mjobs, void* dev_yjobs, cudaStream_t s,
                       cudaEvent_t ev_lists, cudaEvent_t ev_lists2, unsigned ev_flags);
size_t mitm_job_bytes(int nF);
size_t mitm_yjob_bytes(int nF);

// Bytes of one problem's buffers for geometry g (uses g.hcap).
size_t match_bytes(const MatchGeom& g);

// Lay out one problem's buffers inside `ws` (256-byte aligned pieces).
void match_layout(const MatchGeom& g, char* ws, ProbJob* pj);

// Assign grid bases, upload the job arrays (host_halves: 2*np scratch) and
// launch count -> column scan -> bucket scan -> scatter -> join on stream s.
// ev_count / ev_scatter, if given, are recorded after the scans and after
// the scatter.
// All problems of one call use the same layout (all optimistic or all exact);
// the optimistic cursors (bcount, hcount) and the exact halo counts must be
// zeroed by the caller.
// Fused problems (ProbJob::fused) may be mixed in; they run k_mitm after the
// table problems' join (with only fused problems, ev_count and ev_scatter are
// both recorded after their sorted lists are built).  *launches (if given)
// receives the kernel count.
cudaError_t run_match(ProbJob* jobs, int np, ProbJob* dev_jobs, HalfJob* dev_halves,
                      HalfJob* host_halves, cudaStream_t s, cudaEvent_t ev_count, cudaEvent_t ev_scatter,
                      int* launches = nullptr);

}  // namespace rfr
