// runtime.cu — host runtime of the RFR library: context, batch pipeline,
// memory budget, serving queue (continuous batching) and the C ABI of rfr.h.
//
// Pipeline for a batch of polynomials on one stream:
//   validate (monic, range, square-free mod primes)      host
//   H2D coefficients                                     copy
//   K-a roots, K-b weights                               kernels
//   D2H plans -> per-problem table geometry             host (sync 1)
//   K-c/K-d/K-e match for every problem, in sub-batches  kernels
//     that fit the memory budget
//   D2H candidate counts and candidates                  host (sync 2)
//   K-f verify all candidates                            kernel
//   D2H verdicts -> atoms of the verified divisors       host (sync 3)
//   K-f on the atoms, returning their integer polynomials kernel
//   D2H factors -> canonical order                       host (sync 4)
#include "rfr_device.cuh"
#include "k_match.cuh"

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <fstream>
#include <functional>
#include <map>
#include <memory>
#include <sstream>
#include <string>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

extern "C" int rfr_stage_validate(const int64_t*, const int32_t*, int, int32_t*, void*);
extern "C" int rfr_stage_roots(const int64_t*, const int32_t*, int, int, double*, double*, int32_t*, void*);
extern "C" int rfr_stage_weights(const int64_t*, const int32_t*, int, const double*, const double*,
                                 const int32_t*, double, rfr_plan*, void*);
extern "C" int rfr_stage_verify(const int64_t*, const int32_t*, const double*, const rfr_plan*,
                                const int32_t*, const uint64_t*, const uint64_t*, int, int32_t*,
                                int64_t*, void*);

namespace rfr {

// ---------------------------------------------------------------- helpers
struct Bits {
    uint64_t lo = 0, hi = 0;
    bool get(int k) const { return k < 64 ? (lo >> k) & 1 : (hi >> (k - 64)) & 1; }
    void set(int k) { if (k < 64) lo |= 1ull << k; else hi |= 1ull << (k - 64); }
    Bits operator&(const Bits& o) const { return {lo & o.lo, hi & o.hi}; }
    Bits operator~() const { return {~lo, ~hi}; }
    bool operator==(const Bits& o) const { return lo == o.lo && hi == o.hi; }
};
static Bits full_bits(int n) {
    Bits b;
    b.lo = n >= 64 ? ~0ull : (n ? (~0ull >> (64 - n)) : 0ull);
    b.hi = n > 64 ? (~0ull >> (128 - n)) : 0ull;
    return b;
}

// ---------------------------------------------------------------- allocation
struct DevAlloc {
    rfr_alloc_fn fa = nullptr;
    rfr_free_fn ff = nullptr;
    void* user = nullptr;
    void* get(size_t bytes, cudaStream_t s) {
        if (bytes == 0) bytes = 256;
        if (fa) return fa(bytes, user, (void*)s);
        void* p = nullptr;
        if (cudaMallocAsync(&p, bytes, s) != cudaSuccess) { cudaGetLastError(); return nullptr; }
        return p;
    }
    void put(void* p, size_t bytes, cudaStream_t s) {
        if (!p) return;
        if (ff) ff(p, bytes, user, (void*)s);
        else cudaFreeAsync(p, s);
    }
};

struct Item {
    const int64_t* coeffs;
    int degree;
    int status;
    rfr_factors* out;
};

// Where a sub-batch's candidates are gathered (k_compact_desc reads it from the
// match arena, so that a captured graph needs no kernel arguments that change).
struct CompactDesc {
    const uint64_t* cand;             // [np][cap] per-problem candidate buffers
    uint64_t cap;
    const unsigned long long* ctr;    // [np][8] counters
    int np;
    uint64_t* out;                    // [out_cap] compacted candidates
    uint64_t out_cap;
    uint64_t* offs;                   // [np + 1] their offsets
    uint64_t* inl;                    // [INL] the first INL compacted candidates, beside the offsets
};

// Candidates that come back in the same copy as the counters (a sub-batch with
// at most this many needs no second copy and synchronisation).
constexpr uint64_t INL = 512;

// Match arena of a sub-batch of np problems: the compaction descriptor, np
// ProbJob slots, 2 np HalfJob slots, the counters [np][8], the offsets
// [np + 1] and the first INL compacted candidates.  Everything before the
// offsets is uploaded from the host image in one copy (the counters as zeros);
// the counters, offsets and inline candidates come back in one copy.  The
// layout for np fits in the one for any larger np.
struct ArenaLayout { size_t desc, jobs, halves, ctrs, offs, inl, upload, total; };
static ArenaLayout arena_layout(int np) {
    auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
    ArenaLayout L;
    size_t p = 0;
    L.desc = p;   p += a256(sizeof(CompactDesc));
    L.jobs = p;   p += a256((size_t)np * sizeof(ProbJob));
    L.halves = p; p += a256((size_t)2 * np * sizeof(HalfJob));
    L.ctrs = p;   p += (size_t)np * 64;
    L.offs = p;   p += ((size_t)np + 1) * 8;
    L.inl = p;    p += INL * 8;
    L.upload = L.offs;
    L.total = a256(p);
    return L;
}

// Per-problem working state inside a batch.
struct Work {
    int item;                // index into the batch's items
    int slot;                // index into the device arrays
    rfr_plan plan;           // copied back after K-b
    MatchGeom geom;
    bool full_halo = false;
    bool matched = false;
    uint64_t ctr[6] = {0, 0, 0, 0, 0, 0};
    std::vector<uint64_t> cand;
    std::vector<Bits> verified;
    std::vector<Bits> atoms;
    std::vector<std::vector<int64_t>> factors;
    int status = RFR_OK;
};

struct Ctx;

// One pipeline = one stream plus its reusable buffers.
struct Pipeline {
    Ctx* ctx = nullptr;
    cudaStream_t s = nullptr;
    cudaEvent_t ev[10] = {};
    int cap = 0;                      // problems the device arrays hold
    int64_t* d_coeffs = nullptr;
    int32_t* d_deg = nullptr;
    double* d_roots = nullptr;
    double* d_radius = nullptr;
    int32_t* d_rstat = nullptr;
    rfr_plan* d_plans = nullptr;
    int64_t* h_coeffs = nullptr;      // pinned
    int32_t* h_deg = nullptr;         // pinned
    rfr_plan* h_plans = nullptr;      // pinned
    char* h_stage = nullptr;          // pinned staging of counters, candidates and verify jobs
    size_t h_stage_cap = 0;
    // h_stage grown to at least `bytes` (null if pinned memory is short); the
    // stream is idle whenever this is called, so the old buffer is unused
    char* stage(size_t bytes) {
        if (bytes <= h_stage_cap) return h_stage;
        if (h_stage) cudaFreeHost(h_stage);
        h_stage = nullptr;
        h_stage_cap = 0;
        const size_t nb = std::max(bytes, (size_t)1 << 20);
        if (cudaMallocHost(&h_stage, nb) != cudaSuccess) { cudaGetLastError(); h_stage = nullptr; return nullptr; }
        h_stage_cap = nb;
        return h_stage;
    }
    const int64_t* cur_coeffs = nullptr;   // coefficient rows of the running batch (device)
    const int32_t* cur_deg = nullptr;
    // captured prologue graphs (copy in, validate, roots, weights, plans out) per batch shape
    struct PrologueGraph { int B; int mode; double eps; cudaGraphExec_t exec; };
    std::vector<PrologueGraph> graphs;
    // The match arena: a sub-batch's job records, counters, candidate offsets and
    // compaction descriptor (arena_layout), at device addresses that stay fixed
    // until the arena is regrown, and its pinned host image.  A sub-batch of
    // fused problems uploads its records from the image in one copy, so a
    // captured match graph replays with new records and no parameter updates.
    char* d_arena = nullptr;
    char* h_arena = nullptr;
    // captured match graphs (record upload, sorted lists, k_mitm, k_mitm_check,
    // compaction) by launch shape; a shape is captured the second time it
    // occurs, so that shapes that never recur cost no capture
    struct MatchGraph { std::vector<int> key; cudaGraphExec_t exec; uint64_t used; };
    std::vector<MatchGraph> mgraphs;
    std::deque<std::vector<int>> mseen;
    uint64_t mclock = 0;
    uint32_t graph_launches = 0;      // graphs launched by the running batch
    // graphs (prologue and match) for this pipeline's batches: on for caller
    // batches (blocking, device and asynchronous calls), whose shapes recur when
    // a workload does; off for the batches continuous batching forms from the
    // request queue, whose sizes and compositions rarely recur
    bool match_graphs = true;
    void drop_graphs() {
        for (auto& g : graphs) cudaGraphExecDestroy(g.exec);
        graphs.clear();
        for (auto& g : mgraphs) cudaGraphExecDestroy(g.exec);
        mgraphs.clear();
        mseen.clear();
    }
    int issue_prologue(int B, const int64_t* d_co, const int32_t* d_dg, bool copy_in,
                       uint64_t& h2d, uint64_t& d2h, uint32_t& launches, unsigned ev_flags = cudaEventRecordDefault);
    // The match of a sub-batch of np fused problems whose records are in the
    // arena's host image (layout AL, launch shape sh): a replayed graph when
    // the shape has one, else direct launches (capturing the shape on its
    // second occurrence).
    int run_match_graph(const MitmShape& sh, const ArenaLayout& AL, int np);
    // issue(flags) under the graph of `key` (replayed if captured; captured on
    // the key's second occurrence; else launched directly).  issue must only
    // enqueue work on s (it may run under stream capture) and records its
    // events with `flags`.
    int run_graphed(const std::vector<int>& key, const std::function<cudaError_t(unsigned)>& issue);
    bool init(Ctx* c);
    void destroy();
    bool reserve(int n);
    // dev_coeffs/dev_deg: device rows for every item in order (device inputs),
    // or null (host inputs, copied in).
    int run(std::vector<Item>& items, const int64_t* dev_coeffs = nullptr, const int32_t* dev_deg = nullptr);
    // Key-range sharding of the batch (rfr_factor_batch_sharded): the fused
    // match searches only this shard's slabs, other matches run on shard 0
    // (and on any shard that redoes a problem with the table match), and the
    // verified divisor sets of all shards are exchanged through `gather`
    // before the atoms.
    struct Shard { int index = 0, count = 1; rfr_gather_fn gather = nullptr; void* user = nullptr; } shard;
    bool sharded() const { return shard.count > 1; }
};

struct Request {
    uint64_t ticket;
    std::vector<int64_t> coeffs;
    int degree;
    int status = RFR_PENDING;
    bool cancelled = false, running = false, done = false;
    rfr_factors result{};
};

// One whole batch queued by rfr_factor_batch_async: the rows are copied at
// submit; outs / statuses are the caller's, filled by the worker that runs it.
struct BatchJob {
    uint64_t ticket;
    std::vector<int64_t> flat;
    std::vector<const int64_t*> rows;
    std::vector<int> degrees;
    rfr_factors* outs;
    int* statuses;
    int rc = RFR_PENDING;
    bool done = false;
};

struct Ctx {
    rfr_config cfg;
    int device = 0;
    DevAlloc alloc;
    size_t budget = 0;
    std::mutex budget_mu;
    std::condition_variable budget_cv;
    size_t budget_used = 0;
    std::mutex sync_mu;               // serialises rfr_factor / rfr_factor_batch
    Pipeline sync_pipe;
    // serving
    std::mutex q_mu;
    std::condition_variable q_cv, done_cv;
    std::deque<Request*> pending;
    std::unordered_map<uint64_t, Request*> reqs;
    std::deque<BatchJob*> batch_q;                 // whole batches, run before single requests
    std::unordered_map<uint64_t, BatchJob*> batch_jobs;
    uint64_t next_ticket = 1;
    bool stop = false;
    int running_batches = 0;
    std::vector<std::thread> workers;
    int n_workers = 0;                            // set before the first worker starts
    std::vector<std::unique_ptr<Pipeline>> worker_pipes;
    // autotuned layouts per (n_a, n_b)
    std::mutex tune_mu;
    std::map<std::pair<int, int>, TuneParams> tuned;
    std::string tune_path, device_name;

    // Reserve `bytes` of the device budget; waits while other batches hold it.
    // A batch holds at most one reservation at a time and every holder runs to
    // completion, so the wait ends, also while the context is being destroyed
    // (running batches finish normally).
    bool reserve(size_t bytes) {
        std::unique_lock<std::mutex> lk(budget_mu);
        if (bytes > budget) return false;
        budget_cv.wait(lk, [&] { return budget_used + bytes <= budget; });
        budget_used += bytes;
        return true;
    }
    void release(size_t bytes) {
        std::lock_guard<std::mutex> lk(budget_mu);
        budget_used -= bytes;
        budget_cv.notify_all();
    }
};

static int cuda_ok(cudaError_t e) { return e == cudaSuccess ? RFR_OK : RFR_E_CUDA; }

bool Pipeline::init(Ctx* c) {
    ctx = c;
    if (cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) != cudaSuccess) return false;
    for (auto& e : ev) if (cudaEventCreate(&e) != cudaSuccess) return false;
    return true;
}

void Pipeline::destroy() {
    if (s) cudaStreamSynchronize(s);
    drop_graphs();
    auto put = [&](void* p) { if (p) ctx->alloc.put(p, 0, s); };
    put(d_coeffs); put(d_deg); put(d_roots); put(d_radius); put(d_rstat); put(d_plans); put(d_arena);
    if (s) cudaStreamSynchronize(s);
    if (h_coeffs) cudaFreeHost(h_coeffs);
    if (h_deg) cudaFreeHost(h_deg);
    if (h_plans) cudaFreeHost(h_plans);
    if (h_arena) cudaFreeHost(h_arena);
    if (h_stage) cudaFreeHost(h_stage);
    h_stage = nullptr;
    h_stage_cap = 0;
    for (auto& e : ev) if (e) cudaEventDestroy(e);
    if (s) cudaStreamDestroy(s);
    s = nullptr;
}

bool Pipeline::reserve(int n) {
    if (n <= cap) return true;
    int nc = std::max(n, std::max(16, cap * 2));
    cudaStreamSynchronize(s);
    drop_graphs();                      // they name the buffers freed below
    auto put = [&](void* p) { if (p) ctx->alloc.put(p, 0, s); };
    put(d_coeffs); put(d_deg); put(d_roots); put(d_radius); put(d_rstat); put(d_plans); put(d_arena);
    if (h_coeffs) cudaFreeHost(h_coeffs);
    if (h_deg) cudaFreeHost(h_deg);
    if (h_plans) cudaFreeHost(h_plans);
    if (h_arena) cudaFreeHost(h_arena);
    h_arena = nullptr;
    const size_t abytes = arena_layout(nc).total;
    d_arena = (char*)ctx->alloc.get(abytes, s);
    d_coeffs = (int64_t*)ctx->alloc.get((size_t)nc * LDC * 8, s);
    d_deg = (int32_t*)ctx->alloc.get((size_t)nc * 4, s);
    d_roots = (double*)ctx->alloc.get((size_t)nc * DMAX * 32, s);
    d_radius = (double*)ctx->alloc.get((size_t)nc * DMAX * 8, s);
    d_rstat = (int32_t*)ctx->alloc.get((size_t)nc * 4, s);
    d_plans = (rfr_plan*)ctx->alloc.get((size_t)nc * sizeof(rfr_plan), s);
    bool ok = d_coeffs && d_deg && d_roots && d_radius && d_rstat && d_plans && d_arena;
    ok = ok && cudaMallocHost(&h_arena, abytes) == cudaSuccess;
    ok = ok && cudaMallocHost(&h_coeffs, (size_t)nc * LDC * 8) == cudaSuccess;
    ok = ok && cudaMallocHost(&h_deg, (size_t)nc * 4) == cudaSuccess;
    ok = ok && cudaMallocHost(&h_plans, (size_t)nc * sizeof(rfr_plan)) == cudaSuccess;
    cap = ok ? nc : 0;
    return ok;
}

// Candidates of a sub-batch's np problems into one buffer: problem i's
// min(counters[8 i + 2], cap) patterns, from cand[i cap ..), land at
// out[offs[i] ..); offs[np] = their total.  One block (the candidates are few);
// nothing is copied when the total exceeds out_cap (the host then copies
// problem by problem).
__device__ __forceinline__ void compact_cands(const uint64_t* __restrict__ cand, uint64_t cap,
                                              const unsigned long long* __restrict__ ctr, int np,
                                              uint64_t* __restrict__ out, uint64_t out_cap,
                                              uint64_t* __restrict__ offs, uint64_t* __restrict__ inl) {
    if (threadIdx.x == 0) {
        uint64_t o = 0;
        for (int i = 0; i < np; ++i) {
            offs[i] = o;
            const uint64_t n = ctr[8 * i + 2];
            o += n < cap ? n : cap;
        }
        offs[np] = o;
    }
    __syncthreads();
    if (offs[np] > out_cap) return;
    for (int i = 0; i < np; ++i) {
        const uint64_t o = offs[i], n = offs[i + 1] - o;
        for (uint64_t j = threadIdx.x; j < n; j += blockDim.x) {
            const uint64_t v = cand[(uint64_t)i * cap + j];
            out[o + j] = v;
            if (o + j < INL) inl[o + j] = v;
        }
    }
}

__global__ void __launch_bounds__(256) k_compact_cands(const uint64_t* __restrict__ cand, uint64_t cap,
                                                        const unsigned long long* __restrict__ ctr, int np,
                                                        uint64_t* __restrict__ out, uint64_t out_cap,
                                                        uint64_t* __restrict__ offs, uint64_t* __restrict__ inl) {
    compact_cands(cand, cap, ctr, np, out, out_cap, offs, inl);
}

// k_compact_cands for the sub-batch described at d (in the match arena).
__global__ void __launch_bounds__(256) k_compact_desc(const CompactDesc* __restrict__ d) {
    const CompactDesc D = *d;
    compact_cands(D.cand, D.cap, D.ctr, D.np, D.out, D.out_cap, D.offs, D.inl);
}

static double ms_between(cudaEvent_t a, cudaEvent_t b) {
    float ms = 0.f;
    if (cudaEventElapsedTime(&ms, a, b) != cudaSuccess) { cudaGetLastError(); return 0.0; }
    return ms;
}

static void fill_factors(rfr_factors* out, const std::vector<std::vector<int64_t>>& fs) {
    out->n_factors = (int)fs.size();
    size_t tot = 0;
    for (auto& f : fs) tot += f.size();
    out->degrees = (int*)malloc(sizeof(int) * std::max<size_t>(1, fs.size()));
    out->coeffs = (int64_t*)malloc(sizeof(int64_t) * std::max<size_t>(1, tot));
    size_t o = 0;
    for (size_t i = 0; i < fs.size(); ++i) {
        out->degrees[i] = (int)fs[i].size() - 1;
        memcpy(out->coeffs + o, fs[i].data(), fs[i].size() * 8);
        o += fs[i].size();
    }
}

static void canonical_sort(std::vector<std::vector<int64_t>>& fs) {
    std::sort(fs.begin(), fs.end(), [](const std::vector<int64_t>& a, const std::vector<int64_t>& b) {
        if (a.size() != b.size()) return a.size() < b.size();
        for (size_t i = 0; i + 1 < a.size(); ++i) if (a[i] != b[i]) return a[i] < b[i];
        return false;
    });
}

// Candidate CTAs per half: spread about four CTAs per SM over the sub-batch.
static int part_ctas(int h, double share_total_elems, int cta_per_sm = 16) {
    const double target = (double)cta_per_sm * 148.0;
    double want = std::ldexp(1.0, h) * target / std::max(1.0, share_total_elems);
    int c = 1;
    while (c * 2 <= want && c < 512 && ((uint64_t)c * 2 * 64) <= (1ull << h)) c *= 2;
    return c;
}

int Pipeline::issue_prologue(int B, const int64_t* d_co, const int32_t* d_dg, bool copy_in,
                             uint64_t& h2d, uint64_t& d2h, uint32_t& launches, unsigned ev_flags) {
    Ctx& C = *ctx;
    cudaEventRecordWithFlags(ev[0], s, ev_flags);
    int rc = RFR_OK;
    if (copy_in) {
        rc = cuda_ok(cudaMemcpyAsync(d_coeffs, h_coeffs, (size_t)B * LDC * 8, cudaMemcpyHostToDevice, s));
        if (rc == RFR_OK) rc = cuda_ok(cudaMemcpyAsync(d_deg, h_deg, (size_t)B * 4, cudaMemcpyHostToDevice, s));
        h2d += (uint64_t)B * LDC * 8 + (uint64_t)B * 4;
    }
    if (rc == RFR_OK) rc = rfr_stage_validate(d_co, d_dg, B, d_rstat, s);
    if (rc == RFR_OK) rc = rfr_stage_roots(d_co, d_dg, B, C.cfg.root_mode, d_roots, d_radius, d_rstat, s);
    // k_validate; k_aberth (+ k_aberth64 in FP32-bulk mode), k_polish, k_radius
    launches += C.cfg.root_mode == RFR_ROOTS_FP32_BULK ? 5 : 4;
    cudaEventRecordWithFlags(ev[1], s, ev_flags);
    if (rc == RFR_OK) rc = rfr_stage_weights(d_co, d_dg, B, d_roots, d_radius, d_rstat, C.cfg.eps_override, d_plans, s);
    launches += 1;
    cudaEventRecordWithFlags(ev[2], s, ev_flags);
    if (rc == RFR_OK) rc = cuda_ok(cudaMemcpyAsync(h_plans, d_plans, (size_t)B * sizeof(rfr_plan), cudaMemcpyDeviceToHost, s));
    d2h += (uint64_t)B * sizeof(rfr_plan);
    return rc;
}

// Time one problem's match with layout knobs tp: the problem is matched as
// `copies` identical problems in one launch sequence, so that the CTA counts
// and the concurrency resemble a real sub-batch; one warm-up, one timed run.
// Returns milliseconds per problem, or a negative value if it does not fit.
static double time_layout(Ctx& C, cudaStream_t s, const rfr_plan& plan, const rfr_plan* dplan,
                          const TuneParams& tp, cudaEvent_t e0, cudaEvent_t e1) {
    const double elems = std::ldexp(1.0, plan.n_a) + std::ldexp(1.0, plan.n_b);
    MatchGeom g;
    int copies = 8;
    for (; copies >= 1; copies /= 2) {
        auto ctas = [&](int h) {
            double want = std::ldexp(1.0, h) * tp.cta_per_sm * 148.0 / (elems * copies);
            int c = 1;
            while (c * 2 <= want && c < 512) c *= 2;
            return c;
        };
        if (!match_geometry(plan.n_a, plan.n_b, plan.window, ctas(plan.n_a), ctas(plan.n_b), &g, true, &tp)) return -1.0;
        if ((g.bytes + 4096) * (size_t)copies + 4096 <= C.budget / 2) break;
    }
    if (copies < 1) return -1.0;
    const size_t per = ((g.bytes + 255) & ~(size_t)255) + 4096;
    const size_t head = (((size_t)copies * sizeof(ProbJob) + 255) & ~(size_t)255) + (((size_t)2 * copies * sizeof(HalfJob) + 255) & ~(size_t)255);
    const size_t bytes = head + per * copies;
    char* ws = (char*)C.alloc.get(bytes, s);
    if (!ws) return -1.0;
    double best = -1.0;
    std::vector<ProbJob> jobs(copies);
    std::vector<HalfJob> halves(2 * copies);
    ProbJob* d_jobs = (ProbJob*)ws;
    HalfJob* d_halves = (HalfJob*)(ws + (((size_t)copies * sizeof(ProbJob) + 255) & ~(size_t)255));
    for (int rep = 0; rep < 2; ++rep) {
        for (int c = 0; c < copies; ++c) {
            char* base = ws + head + per * c;
            ProbJob& pj = jobs[c];
            memset(&pj, 0, sizeof(pj));
            match_layout(g, base, &pj);
            uint64_t* ctr = (uint64_t*)(base + ((g.bytes + 255) & ~(size_t)255));
            uint64_t* cand = ctr + 32;
            pj.A.w = dplan->w; pj.B.w = dplan->w + plan.n_a;
            pj.w_a = dplan->w; pj.w2_a = dplan->w2; pj.w_b = dplan->w + plan.n_a; pj.w2_b = dplan->w2 + plan.n_a;
            pj.W = plan.window; pj.W2 = plan.window2;
            pj.cand = cand; pj.cap = 256; pj.ctr = (unsigned long long*)ctr;
            pj.A.err = pj.B.err = (int*)(ctr + 4);
            cudaMemsetAsync(ctr, 0, 64, s);
            if (!g.fused) cudaMemsetAsync(pj.A.bcount, 0, 3 * (((((size_t)1 << g.d1) * 4) + 255) & ~(size_t)255), s);
        }
        cudaEventRecord(e0, s);
        if (run_match(jobs.data(), copies, d_jobs, d_halves, halves.data(), s, nullptr, nullptr) != cudaSuccess) break;
        cudaEventRecord(e1, s);
        if (cudaStreamSynchronize(s) != cudaSuccess) break;
        best = ms_between(e0, e1) / copies;
    }
    C.alloc.put(ws, bytes, s);
    cudaGetLastError();
    return best;
}

// Coordinate search over the layout knobs for one (n_a, n_b) class: the key-unit
// size and the bin limit for the fused match, the low-list bits, bucket digit and
// CTAs per SM for the table match.
static TuneParams tune_class(Ctx& C, cudaStream_t s, const rfr_plan& plan, const rfr_plan* dplan,
                             cudaEvent_t e0, cudaEvent_t e1) {
    TuneParams best;
    double tbest = time_layout(C, s, plan, dplan, best, e0, e1);
    if (tbest < 0) return best;
    MatchGeom g0;
    if (match_geometry(plan.n_a, plan.n_b, plan.window, 1, 1, &g0, true) && g0.fused) {
        const int uvals[] = {13, 12}, bvals[] = {12};
        for (int v : uvals) { TuneParams t = best; t.unit_log = v; double m = time_layout(C, s, plan, dplan, t, e0, e1); if (m > 0 && m < tbest) { tbest = m; best = t; } }
        for (int v : bvals) { TuneParams t = best; t.nbl_max = v; double m = time_layout(C, s, plan, dplan, t, e0, e1); if (m > 0 && m < tbest) { tbest = m; best = t; } }
        return best;
    }
    const int lvals[] = {15, 17}, dvals[] = {12}, cvals[] = {8, 32};
    for (int v : lvals) { TuneParams t = best; t.l_max = v; double m = time_layout(C, s, plan, dplan, t, e0, e1); if (m > 0 && m < tbest) { tbest = m; best = t; } }
    for (int v : dvals) { TuneParams t = best; t.d1_off = v; double m = time_layout(C, s, plan, dplan, t, e0, e1); if (m > 0 && m < tbest) { tbest = m; best = t; } }
    for (int v : cvals) { TuneParams t = best; t.cta_per_sm = v; double m = time_layout(C, s, plan, dplan, t, e0, e1); if (m > 0 && m < tbest) { tbest = m; best = t; } }
    return best;
}

static void tune_cache_load(Ctx& C) {
    if (C.tune_path.empty()) return;
    std::ifstream f(C.tune_path);
    std::string line;
    while (std::getline(f, line)) {
        std::istringstream is(line);
        std::string dev;
        int na, nb;
        TuneParams t;
        if (std::getline(is, dev, '\t') && dev == C.device_name &&
            (is >> na >> nb >> t.l_max >> t.d1_off >> t.cta_per_sm >> t.unit_log >> t.nbl_max))
            C.tuned[{na, nb}] = t;
    }
}

static void tune_cache_store(Ctx& C, int na, int nb, const TuneParams& t) {
    if (C.tune_path.empty()) return;
    std::ofstream f(C.tune_path, std::ios::app);
    f << C.device_name << '\t' << na << ' ' << nb << ' ' << t.l_max << ' ' << t.d1_off << ' ' << t.cta_per_sm
      << ' ' << t.unit_log << ' ' << t.nbl_max << '\n';
}

int Pipeline::run_graphed(const std::vector<int>& key, const std::function<cudaError_t(unsigned)>& issue) {
    MatchGraph* g = nullptr;
    for (auto& x : mgraphs) if (x.key == key) g = &x;
    if (!g) {
        auto it = std::find(mseen.begin(), mseen.end(), key);
        if (it == mseen.end()) {                      // first occurrence: launch directly
            mseen.push_back(key);
            if (mseen.size() > 64) mseen.pop_front();
            return cuda_ok(issue(cudaEventRecordDefault));
        }
        mseen.erase(it);
        cudaGraph_t graph = nullptr;
        cudaGraphExec_t exec = nullptr;
        cudaError_t e = cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal);
        if (e == cudaSuccess) {
            const cudaError_t e2 = issue(cudaEventRecordExternal);
            e = cudaStreamEndCapture(s, &graph);
            if (e == cudaSuccess) e = e2;
        }
        if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
        if (graph) cudaGraphDestroy(graph);
        if (e != cudaSuccess) {                       // not captured: launch directly
            cudaGetLastError();
            if (exec) cudaGraphExecDestroy(exec);
            return cuda_ok(issue(cudaEventRecordDefault));
        }
        if (mgraphs.size() >= 16) {                   // evict the least recently used
            auto lru = std::min_element(mgraphs.begin(), mgraphs.end(),
                                        [](const MatchGraph& a, const MatchGraph& b) { return a.used < b.used; });
            cudaGraphExecDestroy(lru->exec);
            mgraphs.erase(lru);
        }
        mgraphs.push_back({key, exec, 0});
        g = &mgraphs.back();
    }
    g->used = ++mclock;
    ++graph_launches;
    return cuda_ok(cudaGraphLaunch(g->exec, s));
}

int Pipeline::run_match_graph(const MitmShape& sh, const ArenaLayout& AL, int np) {
    char* d = d_arena;
    // the launch shape: everything the graph's nodes depend on besides the
    // arena's addresses (fixed until a regrow, which drops the graphs)
    std::vector<int> key{np, sh.nF, sh.nh, sh.ctas, sh.dir_lmax, sh.wrap, sh.wide};
    key.insert(key.end(), sh.ls.begin(), sh.ls.end());
    return run_graphed(key, [&](unsigned flags) -> cudaError_t {
        cudaError_t e = cudaMemcpyAsync(d, h_arena, AL.upload, cudaMemcpyHostToDevice, s);
        if (e == cudaSuccess) e = mitm_issue(sh, d + AL.jobs, d + AL.halves, s, ev[4], ev[5], flags);
        if (e == cudaSuccess) {
            k_compact_desc<<<1, 256, 0, s>>>((const CompactDesc*)(d + AL.desc));
            e = cudaGetLastError();
        }
        return e;
    });
}

int Pipeline::run(std::vector<Item>& items, const int64_t* dev_coeffs, const int32_t* dev_deg) {
    Ctx& C = *ctx;
    const bool timing = C.cfg.timing != 0;
    const bool device_in = dev_coeffs != nullptr;
    auto t_host0 = std::chrono::steady_clock::now();
    uint64_t h2d = 0, d2h = 0;
    uint32_t launches = 0;
    graph_launches = 0;
    std::vector<Work> work;
    // ---- host-side argument checks (host inputs); device inputs are checked by K-v
    for (size_t i = 0; i < items.size(); ++i) {
        Item& it = items[i];
        memset(it.out, 0, sizeof(rfr_factors));
        it.status = RFR_OK;
        if (!device_in) {
            if (!it.coeffs || it.degree < 1 || it.degree > DMAX) { it.status = it.coeffs ? RFR_E_RANGE : RFR_E_INVALID; continue; }
            if (it.coeffs[it.degree] != 1) { it.status = RFR_E_NOT_MONIC; continue; }
            bool range = true;
            for (int k = 0; k <= it.degree; ++k)
                if (it.coeffs[k] >= (1ll << 53) || it.coeffs[k] <= -(1ll << 53)) range = false;
            if (!range) { it.status = RFR_E_RANGE; continue; }
        }
        Work w;
        w.item = (int)i;
        w.slot = (int)work.size();
        w.full_halo = C.cfg.match_path == RFR_MATCH_TABLES;     // tables with the count-pass layout
        work.push_back(std::move(w));
    }
    const int B = (int)work.size();
    if (B == 0) return RFR_OK;
    if (!reserve(B)) return RFR_E_OOM;
    const int64_t* d_co = d_coeffs;
    const int32_t* d_dg = d_deg;
    int rc = RFR_OK;
    if (device_in) {
        d_co = dev_coeffs;                     // rows are the items in order (every item has a slot)
        d_dg = dev_deg;
    } else {
        for (auto& w : work) {
            const Item& it = items[w.item];
            int64_t* row = h_coeffs + (size_t)w.slot * LDC;
            memset(row, 0, LDC * 8);
            memcpy(row, it.coeffs, (it.degree + 1) * 8);
            h_deg[w.slot] = it.degree;
        }
    }
    cur_coeffs = d_co;
    cur_deg = d_dg;
    if (!device_in && C.cfg.use_graphs && match_graphs) {
        // the prologue's shape depends only on B and the root settings: replay a captured graph
        // (caller batches only: the request queue forms batches of every size, and a capture
        // per size costs more than the launches it saves)
        cudaGraphExec_t exec = nullptr;
        for (auto& g : graphs)
            if (g.B == B && g.mode == C.cfg.root_mode && g.eps == C.cfg.eps_override) exec = g.exec;
        if (!exec) {
            uint64_t h0 = 0, d0 = 0;
            uint32_t l0 = 0;
            cudaGraph_t graph = nullptr;
            rc = cuda_ok(cudaStreamBeginCapture(s, cudaStreamCaptureModeThreadLocal));
            if (rc == RFR_OK) {
                const int rc2 = issue_prologue(B, d_co, d_dg, true, h0, d0, l0, cudaEventRecordExternal);
                rc = cuda_ok(cudaStreamEndCapture(s, &graph));
                if (rc == RFR_OK) rc = rc2;
            }
            if (rc == RFR_OK) rc = cuda_ok(cudaGraphInstantiate(&exec, graph, 0));
            if (graph) cudaGraphDestroy(graph);
            if (rc != RFR_OK) { cudaGetLastError(); return rc; }
            graphs.push_back({B, C.cfg.root_mode, C.cfg.eps_override, exec});
        }
        h2d += (uint64_t)B * LDC * 8 + (uint64_t)B * 4;
        d2h += (uint64_t)B * sizeof(rfr_plan);
        launches += C.cfg.root_mode == RFR_ROOTS_FP32_BULK ? 6 : 5;     // the prologue's kernels (as issue_prologue)
        ++graph_launches;
        rc = cuda_ok(cudaGraphLaunch(exec, s));
    } else {
        rc = issue_prologue(B, d_co, d_dg, !device_in, h2d, d2h, launches);
    }
    if (rc == RFR_OK) rc = cuda_ok(cudaStreamSynchronize(s));
    if (rc != RFR_OK) return rc;
    double t_roots = timing ? ms_between(ev[0], ev[1]) : 0, t_weights = timing ? ms_between(ev[1], ev[2]) : 0;
    double t_count = 0, t_scatter = 0, t_match = 0, t_verify = 0;

    // ---- plan the match
    std::vector<int> todo;
    for (auto& w : work) {
        w.plan = h_plans[w.slot];
        if (w.plan.status != RFR_OK) { w.status = w.plan.status; continue; }
        if (w.plan.n <= 1) continue;                      // a single element: irreducible
        if (w.plan.n_b > 32) { w.status = RFR_E_BUDGET; continue; }
        todo.push_back(w.slot);
    }
    const uint64_t cap = std::max<uint64_t>(1, C.cfg.max_candidates);
    // small problems: one fused shared-memory kernel for all of them
    {
        std::vector<int> small, big;
        for (int sl : todo) (work[sl].plan.n_b <= SMALL_MAX_H && work[sl].plan.window < (1ull << 62) ? small : big).push_back(sl);
        todo.swap(big);
        if (sharded() && shard.index != 0) {              // shard 0 matches the small problems
            for (int sl : small) work[sl].matched = true;
            small.clear();
        }
        if (!small.empty()) {
            const int ns = (int)small.size();
            auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
            const uint64_t out_cap = std::min<uint64_t>((uint64_t)ns * cap, 1ull << 18);
            const size_t cb = (size_t)ns * 64 + ((size_t)ns + 1) * 8;      // counters [ns][8], offsets [ns + 1]
            const size_t bytes = a256((size_t)ns * cap * 8) + a256((size_t)out_cap * 8);
            char* ws = (char*)C.alloc.get(bytes, s);
            if (!ws) return RFR_E_OOM;
            // job records, counters and offsets in the match arena (SmallJob records
            // in its ProbJob slots), candidate buffers in the workspace
            static_assert(sizeof(SmallJob) <= sizeof(ProbJob), "a SmallJob fits a ProbJob slot");
            const ArenaLayout AL = arena_layout(ns);
            SmallJob* d_sj = (SmallJob*)(d_arena + AL.jobs);
            unsigned long long* d_ctrs = (unsigned long long*)(d_arena + AL.ctrs);
            uint64_t* d_offs = (uint64_t*)(d_arena + AL.offs);
            uint64_t* d_cands = (uint64_t*)ws;
            uint64_t* d_compact = (uint64_t*)(ws + a256((size_t)ns * cap * 8));
            const bool graphed = C.cfg.use_graphs && match_graphs;
            std::vector<SmallJob> sj(ns);
            for (int i = 0; i < ns; ++i) {
                Work& w = work[small[i]];
                const rfr_plan* dp = d_plans + w.slot;
                sj[i].w_a = dp->w; sj[i].w2_a = dp->w2;
                sj[i].w_b = dp->w + w.plan.n_a; sj[i].w2_b = dp->w2 + w.plan.n_a;
                sj[i].n_a = w.plan.n_a; sj[i].n_b = w.plan.n_b;
                sj[i].W = w.plan.window; sj[i].W2 = w.plan.window2;
                sj[i].cand = d_cands + (size_t)i * cap; sj[i].cap = cap; sj[i].ctr = d_ctrs + 8 * (size_t)i;
            }
            h2d += (uint64_t)ns * sizeof(SmallJob);
            cudaEventRecord(ev[5], s);
            if (graphed) {
                // the records, the compaction's descriptor and zeroed counters go up in
                // one copy from the arena's host image; k_small and the compaction are a
                // replayed graph once the batch's small-problem count has recurred
                const CompactDesc cd{d_cands, cap, d_ctrs, ns, d_compact, out_cap, d_offs, (uint64_t*)(d_arena + AL.inl)};
                memcpy(h_arena + AL.desc, &cd, sizeof(cd));
                memcpy(h_arena + AL.jobs, sj.data(), sizeof(SmallJob) * ns);
                memset(h_arena + AL.ctrs, 0, (size_t)ns * 64);
                rc = cuda_ok(small_attrs());
                if (rc == RFR_OK)
                    rc = run_graphed({-1, ns}, [&](unsigned) -> cudaError_t {
                        cudaError_t e = cudaMemcpyAsync(d_arena, h_arena, AL.upload, cudaMemcpyHostToDevice, s);
                        if (e == cudaSuccess) e = small_issue(d_sj, ns, s);
                        if (e == cudaSuccess) {
                            k_compact_desc<<<1, 256, 0, s>>>((const CompactDesc*)(d_arena + AL.desc));
                            e = cudaGetLastError();
                        }
                        return e;
                    });
                launches += 2;
            } else {
                cudaMemsetAsync(d_ctrs, 0, (size_t)ns * 64, s);
                rc = cuda_ok(run_small(sj.data(), ns, d_sj, s));
                launches += 1;
                if (rc == RFR_OK) {
                    k_compact_cands<<<1, 256, 0, s>>>(d_cands, cap, d_ctrs, ns, d_compact, out_cap, d_offs,
                                                      (uint64_t*)(d_arena + AL.inl));
                    rc = cuda_ok(cudaGetLastError());
                    launches += 1;
                }
            }
            cudaEventRecord(ev[6], s);
            // counters, offsets and the first INL candidates in one copy
            const size_t cbx = cb + INL * 8;
            std::vector<uint64_t> h_ctr(cbx / 8);
            char* hs = stage(cbx);
            if (rc == RFR_OK) rc = cuda_ok(cudaMemcpyAsync(hs ? (void*)hs : (void*)h_ctr.data(), d_ctrs, cbx, cudaMemcpyDeviceToHost, s));
            d2h += cbx;
            if (rc == RFR_OK) rc = cuda_ok(cudaStreamSynchronize(s));
            if (rc == RFR_OK && hs) memcpy(h_ctr.data(), hs, cbx);
            if (timing && rc == RFR_OK) t_match += ms_between(ev[5], ev[6]);
            const uint64_t* h_offs = h_ctr.data() + 8 * (size_t)ns;
            const uint64_t total = rc == RFR_OK ? h_offs[ns] : 0;
            const bool compacted = total <= out_cap;
            char* hc = nullptr;
            if (rc == RFR_OK && compacted && total <= INL) {
                hc = (char*)(h_ctr.data() + cb / 8);          // came back with the counters
            } else if (rc == RFR_OK && compacted && total) {
                hc = stage((size_t)total * 8);
                rc = hc ? cuda_ok(cudaMemcpyAsync(hc, d_compact, total * 8, cudaMemcpyDeviceToHost, s)) : RFR_E_OOM;
                d2h += total * 8;
                if (rc == RFR_OK) rc = cuda_ok(cudaStreamSynchronize(s));
            }
            for (int i = 0; i < ns && rc == RFR_OK; ++i) {
                Work& w = work[small[i]];
                memcpy(w.ctr, &h_ctr[8 * (size_t)i], sizeof(w.ctr));
                if (w.ctr[3] == 0 && shard.index == 0) { w.status = RFR_E_INTERNAL; continue; }
                if (w.ctr[2] > cap) { w.status = RFR_E_CAND_OVERFLOW; continue; }
                w.cand.resize(w.ctr[2]);
                if (w.ctr[2]) {
                    if (compacted) {
                        memcpy(w.cand.data(), hc + h_offs[i] * 8, w.ctr[2] * 8);
                    } else {
                        rc = cuda_ok(cudaMemcpyAsync(w.cand.data(), d_cands + (size_t)i * cap, w.ctr[2] * 8,
                                                     cudaMemcpyDeviceToHost, s));
                        d2h += w.ctr[2] * 8;
                    }
                }
                w.matched = true;
            }
            if (rc == RFR_OK && !compacted) rc = cuda_ok(cudaStreamSynchronize(s));
            C.alloc.put(ws, bytes, s);
            if (rc != RFR_OK) return rc;
        }
    }
    if (C.cfg.autotune && C.cfg.match_path != RFR_MATCH_SPLAT && C.cfg.match_path != RFR_MATCH_PRUNE) {
        for (int sl : todo) {
            Work& w = work[sl];
            const std::pair<int, int> key{w.plan.n_a, w.plan.n_b};
            bool have;
            { std::lock_guard<std::mutex> lk(C.tune_mu); have = C.tuned.count(key) > 0; }
            if (have) continue;
            const TuneParams t = tune_class(C, s, w.plan, d_plans + w.slot, ev[8], ev[9]);
            std::lock_guard<std::mutex> lk(C.tune_mu);
            if (!C.tuned.count(key)) { C.tuned[key] = t; tune_cache_store(C, key.first, key.second, t); }
        }
    }
    auto params_for = [&](const Work& w) {
        std::lock_guard<std::mutex> lk(C.tune_mu);
        auto it = C.tuned.find({w.plan.n_a, w.plan.n_b});
        return it == C.tuned.end() ? TuneParams() : it->second;
    };
    bool one_at_a_time = false;                       // set when a sub-batch's workspace could not be allocated
    while (!todo.empty()) {
        // take a sub-batch that fits this pipeline's share of the budget
        double tot_elems = 0;
        for (int sl : todo) tot_elems += std::ldexp(1.0, work[sl].plan.n_a) + std::ldexp(1.0, work[sl].plan.n_b);
        std::vector<int> sub, rest;
        size_t bytes = 0;
        const size_t share = C.budget / std::max(1, C.cfg.max_inflight);
        // one layout per sub-batch: optimistic first, exact for problems that overflowed it
        const bool exact_round = work[todo[0]].full_halo;
        for (int sl : todo) {
            Work& w = work[sl];
            if (w.full_halo != exact_round) { rest.push_back(sl); continue; }
            MatchGeom g;
            const TuneParams tp = params_for(w);
            if (!match_geometry(w.plan.n_a, w.plan.n_b, w.plan.window, part_ctas(w.plan.n_a, tot_elems, tp.cta_per_sm),
                                part_ctas(w.plan.n_b, tot_elems, tp.cta_per_sm), &g, !w.full_halo, &tp,
                                C.cfg.match_path == RFR_MATCH_SPLAT ? FUSE_SPLAT :
                                C.cfg.match_path == RFR_MATCH_PRUNE ? FUSE_PRUNE : FUSE_AUTO)) { w.status = RFR_E_WINDOW; continue; }
            if (w.full_halo) { g.hcap = 1ull << g.n_b; g.bytes = match_bytes(g); }
            if (sharded() && shard.index != 0 && !g.fused && !w.full_halo) { w.matched = true; continue; }
            const size_t need = g.bytes + (size_t)cap * 8 + 6 * 8 + 512;
            if (need > C.budget) { w.status = RFR_E_BUDGET; continue; }
            if (!sub.empty() && (one_at_a_time || bytes + need > share)) { rest.push_back(sl); continue; }
            w.geom = g;
            bytes += need;
            sub.push_back(sl);
        }
        todo.swap(rest);
        if (sub.empty()) continue;
        if (!C.reserve(bytes)) { for (int sl : sub) work[sl].status = RFR_E_BUDGET; continue; }
        const int np = (int)sub.size();
        // candidates of all problems are compacted into one buffer before they come back
        const uint64_t out_cap = std::min<uint64_t>((uint64_t)np * cap, 1ull << 18);
        const size_t jobs_bytes = (size_t)np * sizeof(ProbJob) + 2 * (size_t)np * sizeof(HalfJob) +
                                  (((size_t)out_cap * 8 + 255) & ~(size_t)255) + 2048;
        char* ws = (char*)C.alloc.get(bytes + jobs_bytes, s);
        if (!ws) {
            C.release(bytes);
            if (np > 1) {                             // retry its problems one at a time: only those whose
                one_at_a_time = true;                 // own tables cannot be allocated end with RFR_E_OOM
                sub.insert(sub.end(), todo.begin(), todo.end());
                todo.swap(sub);
            } else {
                work[sub[0]].status = RFR_E_OOM;
            }
            continue;
        }
        std::vector<ProbJob> jobs(np);
        std::vector<HalfJob> halves(2 * np);
        char* p = ws;
        auto a256 = [](size_t x) { return (x + 255) & ~(size_t)255; };
        // job records, counters [np][8] and the compacted candidates' offsets [np + 1]
        // (copied back together) live in the match arena
        const ArenaLayout AL = arena_layout(np);
        ProbJob* d_jobs = (ProbJob*)(d_arena + AL.jobs);
        HalfJob* d_halves = (HalfJob*)(d_arena + AL.halves);
        unsigned long long* d_ctrs = (unsigned long long*)(d_arena + AL.ctrs);
        uint64_t* d_offs = (uint64_t*)(d_arena + AL.offs);
        uint64_t* d_cands = (uint64_t*)p; p += a256((size_t)np * cap * 8);     // [np][cap]
        uint64_t* d_compact = (uint64_t*)p; p += a256((size_t)out_cap * 8);
        bool all_fused = true;
        for (int i = 0; i < np; ++i) all_fused = all_fused && work[sub[i]].geom.fused;
        const bool graphed = all_fused && C.cfg.use_graphs && match_graphs;
        if (!graphed) cudaMemsetAsync(d_ctrs, 0, (size_t)np * 64, s);
        for (int i = 0; i < np; ++i) {
            Work& w = work[sub[i]];
            ProbJob& pj = jobs[i];
            memset(&pj, 0, sizeof(pj));
            match_layout(w.geom, p, &pj);
            p += w.geom.bytes;
            uint64_t* cbuf = d_cands + (size_t)i * cap;
            uint64_t* ctr = (uint64_t*)(d_ctrs + 8 * (size_t)i);
            const rfr_plan* dp = d_plans + w.slot;
            pj.A.w = dp->w;                     pj.B.w = dp->w + w.plan.n_a;
            pj.w_a = dp->w;                     pj.w2_a = dp->w2;
            pj.w_b = dp->w + w.plan.n_a;        pj.w2_b = dp->w2 + w.plan.n_a;
            pj.W = w.plan.window;               pj.W2 = w.plan.window2;
            pj.shard = shard.index;             pj.nshards = shard.count;
            pj.cand = cbuf;                     pj.cap = cap;
            pj.ctr = (unsigned long long*)ctr;
            pj.A.err = pj.B.err = (int*)(ctr + 4);
            if (w.geom.fused || w.geom.splat || w.geom.prune)
                ;                                       // no tables (the splat arrays are filled by run_splat)
            else if (w.geom.optimistic)
                cudaMemsetAsync(pj.A.bcount, 0, 3 * (((((size_t)1 << w.geom.d1) * 4) + 255) & ~(size_t)255), s);
            else
                cudaMemsetAsync(pj.B.halo_cnt, 0, (((size_t)1 << w.geom.d1) + 1) * 4, s);
        }
        h2d += (uint64_t)np * sizeof(ProbJob) + 2ull * np * sizeof(HalfJob);
        cudaEventRecord(ev[3], s);
        if (graphed) {
            // fused problems only: the records, with the compaction's descriptor and
            // zeroed counters, go up in one copy from the arena's host image, and the
            // launch sequence is a replayed graph once its shape has recurred
            const CompactDesc cd{d_cands, cap, d_ctrs, np, d_compact, out_cap, d_offs, (uint64_t*)(d_arena + AL.inl)};
            memcpy(h_arena + AL.desc, &cd, sizeof(cd));
            memset(h_arena + AL.ctrs, 0, (size_t)np * 64);
            std::vector<const ProbJob*> F(np);
            for (int i = 0; i < np; ++i) F[i] = &jobs[i];
            MitmShape sh;
            rc = cuda_ok(mitm_prepare(F.data(), np, h_arena + AL.jobs, h_arena + AL.halves, &sh));
            if (rc == RFR_OK) rc = run_match_graph(sh, AL, np);
            launches += (uint32_t)mitm_launches(F.data(), np) + 1;
        } else {
            int nl = 0;
            rc = cuda_ok(run_match(jobs.data(), np, d_jobs, d_halves, halves.data(), s, ev[4], ev[5], &nl));
            launches += (uint32_t)nl;
            if (rc == RFR_OK) {
                k_compact_cands<<<1, 256, 0, s>>>(d_cands, cap, d_ctrs, np, d_compact, out_cap, d_offs,
                                                  (uint64_t*)(d_arena + AL.inl));
                rc = cuda_ok(cudaGetLastError());
                launches += 1;
            }
        }
        cudaEventRecord(ev[6], s);
        // counters, offsets and the first INL compacted candidates in one copy
        // (pinned staging when available)
        const size_t cb = (size_t)np * 64 + ((size_t)np + 1) * 8, cbx = cb + INL * 8;
        std::vector<uint64_t> h_ctr(cbx / 8);
        char* hs = stage(cbx);
        if (rc == RFR_OK) rc = cuda_ok(cudaMemcpyAsync(hs ? (void*)hs : (void*)h_ctr.data(), d_ctrs, cbx, cudaMemcpyDeviceToHost, s));
        d2h += cbx;
        if (rc == RFR_OK) rc = cuda_ok(cudaStreamSynchronize(s));
        if (rc == RFR_OK && hs) memcpy(h_ctr.data(), hs, cbx);
        const uint64_t* h_offs = h_ctr.data() + 8 * (size_t)np;
        const uint64_t total = rc == RFR_OK ? h_offs[np] : 0;
        const bool compacted = total <= out_cap;
        if (timing && rc == RFR_OK) {
            t_count += ms_between(ev[3], ev[4]);
            t_scatter += ms_between(ev[4], ev[5]);
            t_match += ms_between(ev[5], ev[6]);
        }
        // all candidates in one copy when they were compacted (none when they came
        // back with the counters), else problem by problem
        char* hc = nullptr;
        if (rc == RFR_OK && compacted && total <= INL) {
            hc = (char*)(h_ctr.data() + cb / 8);
        } else if (rc == RFR_OK && compacted && total) {
            hc = stage((size_t)total * 8);
            rc = hc ? cuda_ok(cudaMemcpyAsync(hc, d_compact, total * 8, cudaMemcpyDeviceToHost, s)) : RFR_E_OOM;
            d2h += total * 8;
            if (rc == RFR_OK) rc = cuda_ok(cudaStreamSynchronize(s));
        }
        for (int i = 0; i < np && rc == RFR_OK; ++i) {
            Work& w = work[sub[i]];
            memcpy(w.ctr, &h_ctr[8 * (size_t)i], sizeof(w.ctr));
            if (w.ctr[4]) { w.full_halo = true; todo.push_back(w.slot); continue; }   // retry with a full halo
            // the empty pattern must match (in the shard that holds key 0, or on a full redo)
            if (w.ctr[3] == 0 && (shard.index == 0 || !w.geom.fused)) { w.status = RFR_E_INTERNAL; continue; }
            if (w.ctr[2] > cap) { w.status = RFR_E_CAND_OVERFLOW; continue; }
            w.cand.resize(w.ctr[2]);
            if (w.ctr[2]) {
                if (compacted) {
                    memcpy(w.cand.data(), hc + h_offs[i] * 8, w.ctr[2] * 8);
                } else {
                    rc = cuda_ok(cudaMemcpyAsync(w.cand.data(), jobs[i].cand, w.ctr[2] * 8, cudaMemcpyDeviceToHost, s));
                    d2h += w.ctr[2] * 8;
                }
            }
            w.matched = true;
        }
        if (rc == RFR_OK && !compacted) rc = cuda_ok(cudaStreamSynchronize(s));
        C.alloc.put(ws, bytes + jobs_bytes, s);
        C.release(bytes);
        if (rc != RFR_OK) return rc;
    }

    // ---- verify candidates, then extract atoms (two K-f passes)
    auto run_verify = [&](std::vector<int32_t>& jp, std::vector<uint64_t>& jlo, std::vector<uint64_t>& jhi,
                          std::vector<int32_t>& res, std::vector<int64_t>* coeffs_out) -> int {
        const int J = (int)jp.size();
        res.assign(J, 0);
        if (J == 0) return RFR_OK;
        const size_t bytes = (size_t)J * (4 + 8 + 8 + 4) + (coeffs_out ? (size_t)J * LDC * 8 : 0) + 1024;
        char* buf = (char*)C.alloc.get(bytes, s);
        if (!buf) return RFR_E_OOM;
        // jobs: [prob J x 4][pad to 16][lo J x 8][hi J x 8], one copy from pinned staging
        const size_t off_lo = (((size_t)J * 4) + 15) & ~(size_t)15, in_bytes = off_lo + (size_t)J * 16;
        int32_t* dp = (int32_t*)buf;
        uint64_t* dlo = (uint64_t*)(buf + off_lo);
        uint64_t* dhi = dlo + J;
        int32_t* dres = (int32_t*)(dhi + J);
        int64_t* dco = coeffs_out ? (int64_t*)(((uintptr_t)(dres + J) + 15) & ~(uintptr_t)15) : nullptr;
        const size_t out_bytes = (size_t)J * 4 + (coeffs_out ? (size_t)J * LDC * 8 : 0);
        char* hs = stage(std::max(in_bytes, out_bytes));
        int r = RFR_OK;
        if (hs) {
            memcpy(hs, jp.data(), (size_t)J * 4);
            memcpy(hs + off_lo, jlo.data(), (size_t)J * 8);
            memcpy(hs + off_lo + (size_t)J * 8, jhi.data(), (size_t)J * 8);
            r = cuda_ok(cudaMemcpyAsync(buf, hs, in_bytes, cudaMemcpyHostToDevice, s));
        } else {
            r = cuda_ok(cudaMemcpyAsync(dp, jp.data(), J * 4, cudaMemcpyHostToDevice, s));
            if (r == RFR_OK) r = cuda_ok(cudaMemcpyAsync(dlo, jlo.data(), J * 8, cudaMemcpyHostToDevice, s));
            if (r == RFR_OK) r = cuda_ok(cudaMemcpyAsync(dhi, jhi.data(), J * 8, cudaMemcpyHostToDevice, s));
        }
        h2d += (uint64_t)J * 20;
        if (r == RFR_OK) r = rfr_stage_verify(d_co, d_dg, d_roots, d_plans, dp, dlo, dhi, J, dres, dco, s);
        launches += 1;
        // results (and coefficients) back through the same staging: the copy in is
        // ordered before them on the stream
        char* ho = hs;
        if (r == RFR_OK) r = cuda_ok(cudaMemcpyAsync(ho ? (void*)ho : (void*)res.data(), dres, J * 4, cudaMemcpyDeviceToHost, s));
        d2h += (uint64_t)J * 4;
        if (r == RFR_OK && coeffs_out) {
            coeffs_out->resize((size_t)J * LDC);
            r = cuda_ok(cudaMemcpyAsync(ho ? (void*)(ho + (size_t)J * 4) : (void*)coeffs_out->data(), dco,
                                        (size_t)J * LDC * 8, cudaMemcpyDeviceToHost, s));
            d2h += (uint64_t)J * LDC * 8;
        }
        if (r == RFR_OK) r = cuda_ok(cudaStreamSynchronize(s));
        if (r == RFR_OK && ho) {
            memcpy(res.data(), ho, (size_t)J * 4);
            if (coeffs_out) memcpy(coeffs_out->data(), ho + (size_t)J * 4, (size_t)J * LDC * 8);
        }
        C.alloc.put(buf, bytes, s);
        return r;
    };
    cudaEventRecord(ev[7], s);
    {
        std::vector<int32_t> jp, res;
        std::vector<uint64_t> jlo, jhi;
        std::vector<int> owner;
        for (auto& w : work) {
            if (w.status != RFR_OK || !w.matched) continue;
            for (size_t c = 0; c < w.cand.size(); ++c) {
                jp.push_back(w.slot);
                jlo.push_back(w.cand[c]);                // patterns over elements 0..n-2 (n-1 <= 64)
                jhi.push_back(0);
                owner.push_back(w.slot);
            }
        }
        rc = run_verify(jp, jlo, jhi, res, nullptr);
        if (rc != RFR_OK) return rc;
        for (size_t j = 0; j < res.size(); ++j) {
            Work& w = work[owner[j]];
            if (res[j] == 1) { Bits b; b.lo = jlo[j]; w.verified.push_back(b); }
            else if (res[j] == RFR_E_OVERFLOW) w.status = RFR_E_OVERFLOW;
        }
    }
    if (sharded()) {
        // every shard's verified divisor sets, as (item, lo, hi) triples
        std::vector<uint64_t> mine;
        for (auto& w : work)
            for (auto& v : w.verified) { mine.push_back((uint64_t)w.item); mine.push_back(v.lo); mine.push_back(v.hi); }
        uint64_t* all = nullptr;
        size_t n_all = 0;
        if (!shard.gather || shard.gather(mine.data(), mine.size() / 3, &all, &n_all, shard.user) != 0)
            { free(all); return RFR_E_INVALID; }
        std::vector<int> by_item(items.size(), -1);
        for (auto& w : work) by_item[w.item] = w.slot;
        for (size_t t = 0; t < n_all; ++t) {
            const uint64_t it = all[3 * t];
            if (it >= items.size() || by_item[it] < 0) continue;
            Work& w = work[by_item[it]];
            const Bits b{all[3 * t + 1], all[3 * t + 2]};
            bool seen = false;
            for (auto& x : w.verified) if (x == b) { seen = true; break; }
            if (!seen) w.verified.push_back(b);
        }
        free(all);
    }
    {
        std::vector<int32_t> jp, res;
        std::vector<uint64_t> jlo, jhi;
        std::vector<std::pair<int, int>> owner;
        for (auto& w : work) {
            if (w.status != RFR_OK) continue;
            const int n = w.plan.n;
            const Bits full = full_bits(n);
            if (n > 1 && !w.verified.empty()) {
                std::vector<Bits> fam;
                fam.push_back(full);
                for (auto& v : w.verified) { fam.push_back(v); fam.push_back(full & ~v); }
                for (int i = 0; i < n; ++i) {
                    Bits a = full;
                    for (auto& t : fam) if (t.get(i)) a = a & t;
                    bool seen = false;
                    for (auto& x : w.atoms) if (x == a) { seen = true; break; }
                    if (!seen) w.atoms.push_back(a);
                }
            } else {
                w.atoms.assign(1, full);                  // irreducible: the single atom is p
            }
            if (w.atoms.size() < 2 && !device_in) continue;   // host inputs: p is known on the host
            for (size_t a = 0; a < w.atoms.size(); ++a) {
                jp.push_back(w.slot); jlo.push_back(w.atoms[a].lo); jhi.push_back(w.atoms[a].hi);
                owner.push_back({w.slot, (int)a});
            }
        }
        std::vector<int64_t> co;
        rc = run_verify(jp, jlo, jhi, res, &co);
        if (rc != RFR_OK) return rc;
        for (size_t j = 0; j < res.size(); ++j) {
            Work& w = work[owner[j].first];
            if (res[j] != 1) { if (w.status == RFR_OK) w.status = res[j] == RFR_E_OVERFLOW ? RFR_E_OVERFLOW : RFR_E_INTERNAL; continue; }
            int e = 0;
            const Bits& a = w.atoms[owner[j].second];
            for (int k = 0; k < w.plan.n; ++k) if (a.get(k)) e += w.plan.kind[k];
            const int64_t* src = co.data() + j * LDC;
            w.factors.emplace_back(src, src + e + 1);
        }
    }
    cudaEventRecord(ev[8], s);
    cudaEventSynchronize(ev[8]);
    if (timing) t_verify = ms_between(ev[7], ev[8]);
    const double t_dev = timing ? ms_between(ev[0], ev[8]) : 0.0;

    // ---- results: factor lists (host inputs: checked exactly against p), then
    // the diagnostics, whose host total covers this phase too
    for (auto& w : work) {
        Item& it = items[w.item];
        if (w.status != RFR_OK) continue;
        std::vector<std::vector<int64_t>> fs;
        if (!w.factors.empty()) fs = std::move(w.factors);
        else fs.emplace_back(it.coeffs, it.coeffs + it.degree + 1);
        if (!device_in && fs.size() > 1) {
            // the product of the factors equals p
            std::vector<__int128> prod(fs[0].begin(), fs[0].end());
            for (size_t f = 1; f < fs.size(); ++f) {
                std::vector<__int128> nx(prod.size() + fs[f].size() - 1, 0);
                for (size_t i = 0; i < prod.size(); ++i)
                    for (size_t j = 0; j < fs[f].size(); ++j) nx[i + j] += prod[i] * (__int128)fs[f][j];
                prod.swap(nx);
            }
            bool same = (int)prod.size() == it.degree + 1;
            for (int k = 0; same && k <= it.degree; ++k) same = prod[k] == (__int128)it.coeffs[k];
            if (!same) { w.status = RFR_E_INTERNAL; continue; }
        }
        canonical_sort(fs);
        fill_factors(it.out, fs);
    }
    const double t_host = std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_host0).count();
    for (auto& w : work) {
        Item& it = items[w.item];
        rfr_diag& dg = it.out->diag;
        dg.n = w.plan.n; dg.r = w.plan.r; dg.c = w.plan.c; dg.n_a = w.plan.n_a; dg.n_b = w.plan.n_b;
        dg.window = w.plan.window;
        dg.half_sums = w.plan.n > 1 ? (1ull << w.plan.n_a) + (1ull << w.plan.n_b) : 0;
        dg.cand_coarse = w.ctr[0]; dg.cand_pre = w.ctr[1]; dg.cand_post = w.ctr[2];
        dg.verified = w.verified.size();
        dg.max_rel_residual = w.plan.max_rel_residual;
        dg.max_root_err = w.plan.max_radius;
        dg.stage_us[0] = t_roots * 1e3; dg.stage_us[1] = t_weights * 1e3; dg.stage_us[2] = t_count * 1e3;
        dg.stage_us[3] = t_scatter * 1e3; dg.stage_us[4] = t_match * 1e3; dg.stage_us[5] = t_verify * 1e3;
        dg.stage_us[6] = t_dev * 1e3; dg.stage_us[7] = t_host * 1e3;
        dg.h2d_bytes = h2d; dg.d2h_bytes = d2h; dg.launches = launches; dg.batch_size = (uint32_t)B;
        dg.graphs = graph_launches;
        if (w.status != RFR_OK) it.status = w.status;
    }
    return RFR_OK;
}

// ---------------------------------------------------------------- serving
// Run a queued whole batch on this worker's pipeline.
static void run_batch_job(Ctx* C, Pipeline* P, BatchJob* J) {
    const int n = (int)J->rows.size();
    std::vector<Item> items(n);
    for (int i = 0; i < n; ++i) items[i] = {J->rows[i], J->degrees[i], RFR_OK, &J->outs[i]};
    P->match_graphs = true;
    const int rc = n ? P->run(items) : RFR_OK;
    for (int i = 0; i < n; ++i) {
        const int st = rc == RFR_OK ? items[i].status : rc;
        if (J->statuses) J->statuses[i] = st;
        if (st != RFR_OK) rfr_factors_free(&J->outs[i]);
    }
    std::lock_guard<std::mutex> lk(C->q_mu);
    J->rc = rc;
    J->done = true;
    --C->running_batches;
}

static void worker_loop(Ctx* C, Pipeline* P) {
    cudaSetDevice(C->device);
    for (;;) {
        std::vector<Request*> batch;
        BatchJob* job = nullptr;
        {
            std::unique_lock<std::mutex> lk(C->q_mu);
            C->q_cv.wait(lk, [&] { return C->stop || !C->pending.empty() || !C->batch_q.empty(); });
            if (C->stop) return;
            if (!C->batch_q.empty()) {
                job = C->batch_q.front();
                C->batch_q.pop_front();
                ++C->running_batches;
            }
        }
        if (job) {
            run_batch_job(C, P, job);
            C->done_cv.notify_all();
            continue;
        }
        {
            std::unique_lock<std::mutex> lk(C->q_mu);
            if (C->stop) return;
            // this worker's share of the queue: the idle workers (this one included)
            // split it, so that a burst is spread over them instead of one worker
            // taking it all while the others wait; a long queue still fills
            // batches of max_batch
            const int idle = std::max(1, C->n_workers - C->running_batches);
            const int share = (int)std::min<size_t>((size_t)C->cfg.max_batch, (C->pending.size() + idle - 1) / idle);
            while (!C->pending.empty() && (int)batch.size() < share) {
                Request* r = C->pending.front();
                C->pending.pop_front();
                if (r->cancelled) continue;
                r->running = true;
                batch.push_back(r);
            }
            ++C->running_batches;
        }
        std::vector<Item> items(batch.size());
        for (size_t i = 0; i < batch.size(); ++i)
            items[i] = {batch[i]->coeffs.data(), batch[i]->degree, RFR_OK, &batch[i]->result};
        P->match_graphs = false;
        int rc = batch.empty() ? RFR_OK : P->run(items);
        {
            std::lock_guard<std::mutex> lk(C->q_mu);
            for (size_t i = 0; i < batch.size(); ++i) {
                batch[i]->status = rc == RFR_OK ? items[i].status : rc;
                batch[i]->running = false;
                batch[i]->done = true;
            }
            --C->running_batches;
        }
        C->done_cv.notify_all();
    }
}

}  // namespace rfr

using namespace rfr;

struct rfr_ctx { Ctx c; };

extern "C" {

const char* rfr_version(void) { return "rfr-b300 0.1 (sm_103a)"; }

const char* rfr_strerror(int st) {
    switch (st) {
        case RFR_OK: return "ok";
        case RFR_PENDING: return "pending";
        case RFR_E_INVALID: return "invalid argument";
        case RFR_E_NOT_MONIC: return "polynomial is not monic";
        case RFR_E_RANGE: return "degree or coefficient out of range";
        case RFR_E_NOT_SQUAREFREE: return "polynomial is not square-free";
        case RFR_E_NO_CONVERGENCE: return "root iteration did not converge";
        case RFR_E_ROOTS: return "roots could not be separated or classified";
        case RFR_E_WINDOW: return "integrality window too wide";
        case RFR_E_CAND_OVERFLOW: return "too many candidate patterns";
        case RFR_E_OVERFLOW: return "integer overflow in exact verification";
        case RFR_E_OOM: return "out of memory";
        case RFR_E_BUDGET: return "tables exceed the memory budget";
        case RFR_E_TIMEOUT: return "timed out";
        case RFR_E_CUDA: return "CUDA error";
        case RFR_E_CANCELLED: return "cancelled";
        case RFR_E_INTERNAL: return "internal consistency check failed";
        default: return "unknown status";
    }
}

int rfr_config_default(rfr_config* cfg) {
    if (!cfg) return RFR_E_INVALID;
    memset(cfg, 0, sizeof(*cfg));
    cfg->device = 0;
    cfg->mem_budget_bytes = 0;
    cfg->max_inflight = 2;
    cfg->max_batch = 64;
    cfg->root_mode = RFR_ROOTS_FP32_BULK;
    cfg->timing = 0;
    cfg->max_candidates = 1ull << 16;
    cfg->eps_override = 0.0;
    cfg->use_graphs = 1;
    cfg->autotune = 0;
    cfg->tune_cache_path = nullptr;
    cfg->match_path = RFR_MATCH_AUTO;
    return RFR_OK;
}

int rfr_create(const rfr_config* cfg_in, rfr_ctx** out) {
    if (!out) return RFR_E_INVALID;
    *out = nullptr;
    rfr_config cfg;
    if (cfg_in) cfg = *cfg_in; else rfr_config_default(&cfg);
    if (cfg.max_inflight < 1 || cfg.max_batch < 1 || (cfg.root_mode != RFR_ROOTS_FP64 && cfg.root_mode != RFR_ROOTS_FP32_BULK) ||
        (cfg.match_path < RFR_MATCH_AUTO || cfg.match_path > RFR_MATCH_PRUNE))
        return RFR_E_INVALID;
    int ndev = 0;
    if (cudaGetDeviceCount(&ndev) != cudaSuccess || cfg.device < 0 || cfg.device >= ndev) { cudaGetLastError(); return RFR_E_CUDA; }
    if (cudaSetDevice(cfg.device) != cudaSuccess) return RFR_E_CUDA;
    rfr_ctx* x = new (std::nothrow) rfr_ctx();
    if (!x) return RFR_E_OOM;
    Ctx& C = x->c;
    C.cfg = cfg;
    C.device = cfg.device;
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    C.budget = cfg.mem_budget_bytes ? cfg.mem_budget_bytes : (size_t)(fr * 0.85);
    {
        cudaDeviceProp prop;
        if (cudaGetDeviceProperties(&prop, cfg.device) == cudaSuccess) C.device_name = prop.name;
        if (cfg.tune_cache_path) C.tune_path = cfg.tune_cache_path;
        C.cfg.tune_cache_path = nullptr;        // the caller's string is not kept
        tune_cache_load(C);
    }
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, cfg.device) == cudaSuccess) {
        uint64_t thr = UINT64_MAX;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    if (!C.sync_pipe.init(&C)) { delete x; return RFR_E_CUDA; }
    for (int i = 0; i < cfg.max_inflight; ++i) {
        C.worker_pipes.emplace_back(new Pipeline());
        if (!C.worker_pipes.back()->init(&C)) { rfr_destroy(x); return RFR_E_CUDA; }
    }
    C.n_workers = cfg.max_inflight;
    C.workers.reserve(cfg.max_inflight);
    for (int i = 0; i < cfg.max_inflight; ++i) C.workers.emplace_back(worker_loop, &C, C.worker_pipes[i].get());
    *out = x;
    return RFR_OK;
}

int rfr_destroy(rfr_ctx* x) {
    if (!x) return RFR_OK;
    Ctx& C = x->c;
    {
        std::lock_guard<std::mutex> lk(C.q_mu);
        C.stop = true;
        for (Request* r : C.pending) { r->status = RFR_E_CANCELLED; r->done = true; }
        C.pending.clear();
        for (BatchJob* J : C.batch_q) {               // queued batches that never ran
            for (size_t i = 0; i < J->rows.size(); ++i) {
                memset(&J->outs[i], 0, sizeof(rfr_factors));
                if (J->statuses) J->statuses[i] = RFR_E_CANCELLED;
            }
            J->rc = RFR_E_CANCELLED;
            J->done = true;
        }
        C.batch_q.clear();
    }
    { std::lock_guard<std::mutex> lk(C.budget_mu); }
    C.budget_cv.notify_all();
    C.q_cv.notify_all();
    for (auto& t : C.workers) t.join();
    for (auto& p : C.worker_pipes) p->destroy();
    C.sync_pipe.destroy();
    for (auto& kv : C.reqs) { rfr_factors_free(&kv.second->result); delete kv.second; }
    for (auto& kv : C.batch_jobs) delete kv.second;
    delete x;
    return RFR_OK;
}

int rfr_set_allocator(rfr_ctx* x, rfr_alloc_fn a, rfr_free_fn f, void* user) {
    if (!x || ((a == nullptr) != (f == nullptr))) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::lock_guard<std::mutex> lk1(C.sync_mu);
    std::lock_guard<std::mutex> lk2(C.q_mu);
    if (C.running_batches || !C.pending.empty()) return RFR_E_INVALID;
    // buffers owned by pipelines were made with the previous allocator: drop them
    auto reset = [&](Pipeline& P) {
        cudaStreamSynchronize(P.s);
        auto put = [&](void* p) { if (p) C.alloc.put(p, 0, P.s); };
        put(P.d_coeffs); put(P.d_deg); put(P.d_roots); put(P.d_radius); put(P.d_rstat); put(P.d_plans); put(P.d_arena);
        cudaStreamSynchronize(P.s);
        P.d_coeffs = nullptr; P.d_deg = nullptr; P.d_roots = nullptr; P.d_radius = nullptr; P.d_rstat = nullptr; P.d_plans = nullptr;
        P.d_arena = nullptr;
        if (P.h_coeffs) cudaFreeHost(P.h_coeffs);
        if (P.h_deg) cudaFreeHost(P.h_deg);
        if (P.h_plans) cudaFreeHost(P.h_plans);
        if (P.h_arena) cudaFreeHost(P.h_arena);
        P.h_coeffs = nullptr; P.h_deg = nullptr; P.h_plans = nullptr; P.h_arena = nullptr;
        P.cap = 0;
        P.drop_graphs();
    };
    reset(C.sync_pipe);
    for (auto& p : C.worker_pipes) reset(*p);
    C.alloc.fa = a; C.alloc.ff = f; C.alloc.user = user;
    return RFR_OK;
}

int rfr_factor_batch(rfr_ctx* x, int count, const int64_t* const* coeffs, const int* degrees,
                     rfr_factors* outs, int* statuses) {
    if (!x || count < 0 || (count && (!coeffs || !degrees || !outs))) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::lock_guard<std::mutex> lk(C.sync_mu);
    cudaSetDevice(C.device);
    std::vector<Item> items(count);
    for (int i = 0; i < count; ++i) items[i] = {coeffs[i], degrees[i], RFR_OK, &outs[i]};
    int rc = C.sync_pipe.run(items);
    for (int i = 0; i < count; ++i) {
        const int st = rc == RFR_OK ? items[i].status : rc;
        if (statuses) statuses[i] = st;
        if (st != RFR_OK) { rfr_factors_free(&outs[i]); }
    }
    return rc;
}

int rfr_factor_batch_sharded(rfr_ctx* x, int count, const int64_t* const* coeffs, const int* degrees,
                             int shard, int nshards, rfr_gather_fn gather, void* user,
                             rfr_factors* outs, int* statuses) {
    if (!x || count < 0 || (count && (!coeffs || !degrees || !outs))) return RFR_E_INVALID;
    if (nshards < 1 || shard < 0 || shard >= nshards || (nshards > 1 && !gather)) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::lock_guard<std::mutex> lk(C.sync_mu);
    cudaSetDevice(C.device);
    std::vector<Item> items(count);
    for (int i = 0; i < count; ++i) items[i] = {coeffs[i], degrees[i], RFR_OK, &outs[i]};
    C.sync_pipe.shard = {shard, nshards, gather, user};
    int rc = C.sync_pipe.run(items);
    C.sync_pipe.shard = Pipeline::Shard();
    for (int i = 0; i < count; ++i) {
        const int st = rc == RFR_OK ? items[i].status : rc;
        if (statuses) statuses[i] = st;
        if (st != RFR_OK) { rfr_factors_free(&outs[i]); }
    }
    return rc;
}

int rfr_factor_batch_device(rfr_ctx* x, int count, const int64_t* d_coeffs, const int32_t* d_degrees,
                            rfr_factors* outs, int* statuses) {
    if (!x || count < 0 || (count && (!d_coeffs || !d_degrees || !outs))) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::lock_guard<std::mutex> lk(C.sync_mu);
    cudaSetDevice(C.device);
    std::vector<Item> items(count);
    for (int i = 0; i < count; ++i) items[i] = {nullptr, 0, RFR_OK, &outs[i]};
    int rc = C.sync_pipe.run(items, d_coeffs, d_degrees);
    for (int i = 0; i < count; ++i) {
        const int st = rc == RFR_OK ? items[i].status : rc;
        if (statuses) statuses[i] = st;
        if (st != RFR_OK) rfr_factors_free(&outs[i]);
    }
    return rc;
}

int rfr_factor_batch_async(rfr_ctx* x, int count, const int64_t* const* coeffs, const int* degrees,
                           rfr_factors* outs, int* statuses, uint64_t* ticket) {
    if (!x || !ticket || count < 0 || (count && (!coeffs || !degrees || !outs))) return RFR_E_INVALID;
    Ctx& C = x->c;
    if (C.n_workers == 0) return RFR_E_INVALID;
    static const int64_t k_unread = 0;              // rows rejected by degree alone are never read
    auto* J = new BatchJob;
    J->outs = outs;
    J->statuses = statuses;
    J->degrees.assign(degrees, degrees + count);
    size_t tot = 0;
    for (int i = 0; i < count; ++i)
        if (coeffs[i] && degrees[i] >= 1 && degrees[i] <= DMAX) tot += (size_t)degrees[i] + 1;
    J->flat.resize(tot);
    J->rows.resize(count);
    size_t o = 0;
    for (int i = 0; i < count; ++i) {
        memset(&outs[i], 0, sizeof(rfr_factors));
        if (statuses) statuses[i] = RFR_PENDING;
        if (!coeffs[i]) { J->rows[i] = nullptr; continue; }
        if (degrees[i] < 1 || degrees[i] > DMAX) { J->rows[i] = &k_unread; continue; }
        memcpy(J->flat.data() + o, coeffs[i], ((size_t)degrees[i] + 1) * 8);
        J->rows[i] = J->flat.data() + o;
        o += (size_t)degrees[i] + 1;
    }
    {
        std::lock_guard<std::mutex> lk(C.q_mu);
        if (C.stop) { delete J; return RFR_E_INVALID; }
        J->ticket = C.next_ticket++;
        C.batch_jobs[J->ticket] = J;
        C.batch_q.push_back(J);
        *ticket = J->ticket;
    }
    C.q_cv.notify_one();
    return RFR_OK;
}

int rfr_batch_wait(rfr_ctx* x, uint64_t ticket, int timeout_ms) {
    if (!x) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::unique_lock<std::mutex> lk(C.q_mu);
    auto it = C.batch_jobs.find(ticket);
    if (it == C.batch_jobs.end()) return RFR_E_INVALID;
    BatchJob* J = it->second;
    auto pred = [&] { return J->done; };
    if (timeout_ms < 0) C.done_cv.wait(lk, pred);
    else if (!C.done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return RFR_E_TIMEOUT;
    const int rc = J->rc;
    C.batch_jobs.erase(ticket);
    delete J;
    return rc;
}

int rfr_factor(rfr_ctx* x, const int64_t* coeffs, int degree, rfr_factors* out) {
    if (!x || !coeffs || !out) return RFR_E_INVALID;
    int st = RFR_OK;
    const int64_t* c[1] = {coeffs};
    int rc = rfr_factor_batch(x, 1, c, &degree, out, &st);
    return rc == RFR_OK ? st : rc;
}

int rfr_submit(rfr_ctx* x, const int64_t* coeffs, int degree, uint64_t* ticket) {
    if (!x || !coeffs || !ticket) return RFR_E_INVALID;
    if (degree < 1 || degree > DMAX) return RFR_E_RANGE;
    if (coeffs[degree] != 1) return RFR_E_NOT_MONIC;
    for (int k = 0; k <= degree; ++k)
        if (coeffs[k] >= (1ll << 53) || coeffs[k] <= -(1ll << 53)) return RFR_E_RANGE;
    Ctx& C = x->c;
    Request* r = new (std::nothrow) Request();
    if (!r) return RFR_E_OOM;
    r->coeffs.assign(coeffs, coeffs + degree + 1);
    r->degree = degree;
    {
        std::lock_guard<std::mutex> lk(C.q_mu);
        if (C.stop) { delete r; return RFR_E_CANCELLED; }
        r->ticket = C.next_ticket++;
        C.reqs[r->ticket] = r;
        C.pending.push_back(r);
        *ticket = r->ticket;
    }
    C.q_cv.notify_one();
    return RFR_OK;
}

static int take_result(Ctx& C, std::unordered_map<uint64_t, Request*>::iterator it, rfr_factors* out) {
    Request* r = it->second;
    const int st = r->status;
    if (out) { *out = r->result; } else rfr_factors_free(&r->result);
    memset(&r->result, 0, sizeof(r->result));
    C.reqs.erase(it);
    delete r;
    return st;
}

int rfr_poll(rfr_ctx* x, uint64_t ticket, rfr_factors* out) {
    if (!x) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::lock_guard<std::mutex> lk(C.q_mu);
    auto it = C.reqs.find(ticket);
    if (it == C.reqs.end()) return RFR_E_INVALID;
    if (!it->second->done) return RFR_PENDING;
    return take_result(C, it, out);
}

int rfr_poll_batch(rfr_ctx* x, int n, const uint64_t* tickets, rfr_factors* outs, int* statuses) {
    if (!x || n < 0 || (n && (!tickets || !outs || !statuses))) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::lock_guard<std::mutex> lk(C.q_mu);
    for (int i = 0; i < n; ++i) {
        auto it = C.reqs.find(tickets[i]);
        if (it == C.reqs.end()) statuses[i] = RFR_E_INVALID;
        else if (!it->second->done) statuses[i] = RFR_PENDING;
        else statuses[i] = take_result(C, it, &outs[i]);
    }
    return RFR_OK;
}

int rfr_wait(rfr_ctx* x, uint64_t ticket, int timeout_ms, rfr_factors* out) {
    if (!x) return RFR_E_INVALID;
    Ctx& C = x->c;
    std::unique_lock<std::mutex> lk(C.q_mu);
    auto it = C.reqs.find(ticket);
    if (it == C.reqs.end()) return RFR_E_INVALID;
    Request* r = it->second;
    auto pred = [&] { return r->done; };
    if (timeout_ms < 0) C.done_cv.wait(lk, pred);
    else if (!C.done_cv.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred)) return RFR_E_TIMEOUT;
    it = C.reqs.find(ticket);
    return take_result(C, it, out);
}

int rfr_cancel(rfr_ctx* x, uint64_t ticket) {
    if (!x) return RFR_E_INVALID;
    Ctx& C = x->c;
    {
        std::lock_guard<std::mutex> lk(C.q_mu);
        auto it = C.reqs.find(ticket);
        if (it == C.reqs.end()) return RFR_E_INVALID;
        Request* r = it->second;
        if (r->done) return RFR_OK;
        if (r->running) return RFR_PENDING;
        r->cancelled = true;
        r->status = RFR_E_CANCELLED;
        r->done = true;
        C.pending.erase(std::remove(C.pending.begin(), C.pending.end(), r), C.pending.end());
    }
    C.done_cv.notify_all();
    return RFR_OK;
}

void rfr_factors_free(rfr_factors* f) {
    if (!f) return;
    free(f->degrees);
    free(f->coeffs);
    f->degrees = nullptr;
    f->coeffs = nullptr;
    f->n_factors = 0;
}

void rfr_factors_free_n(rfr_factors* f, int count) {
    if (!f) return;
    for (int i = 0; i < count; ++i) rfr_factors_free(&f[i]);
}

int64_t rfr_factors_flatten(rfr_factors* f, int count, int64_t* coeffs, size_t coeffs_cap,
                            int32_t* degrees, size_t degrees_cap, int32_t* n_factors) {
    if (count < 0 || (count && (!f || !n_factors))) return RFR_E_INVALID;
    size_t nc = 0, nd = 0;
    for (int i = 0; i < count; ++i) {
        n_factors[i] = f[i].n_factors;
        size_t off = 0;                                   // within result i's coefficients
        for (int k = 0; k < f[i].n_factors; ++k) {
            const size_t len = (size_t)f[i].degrees[k] + 1;
            if (nd + 1 > degrees_cap || nc + len > coeffs_cap) return RFR_E_RANGE;
            degrees[nd++] = f[i].degrees[k];
            memcpy(coeffs + nc, f[i].coeffs + off, len * 8);
            nc += len;
            off += len;
        }
    }
    return (int64_t)nc;
}

}  // extern "C"
