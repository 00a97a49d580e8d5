// k_validate.cu — K-v: input checks on the device (monic, |a_i| < 2^53,
// square-free modulo primes) for inputs that are already in device memory.
//
// One CTA per polynomial.  gcd(p, p') is computed over F_l for the Mersenne
// primes l = 2^31 - 1 and l = 2^61 - 1 by Euclid with pseudo-division
// (a <- lc(b) a - lc(a) x^k b, no inverses), one coefficient per thread.  A
// constant gcd modulo either prime proves p square-free over Q.  Otherwise
// the polynomial is only marked suspect (status RFR_SF_SUSPECT): square-free
// is then decided by the root stage, whose pairwise disjoint inclusion discs
// prove distinct roots, and a failure there is reported as not square-free.
#include "rfr_device.cuh"

namespace rfr {

__device__ __forceinline__ uint64_t mred61(unsigned __int128 x) {
    const uint64_t L = (1ull << 61) - 1;
    uint64_t lo = (uint64_t)x & L;
    uint64_t hi = (uint64_t)(x >> 61);
    uint64_t s = lo + hi;                      // < 2^62 + 2^67? hi < 2^67 only if x < 2^128: fold again
    s = (s & L) + (s >> 61);
    return s >= L ? s - L : s;
}
__device__ __forceinline__ uint64_t mred31(uint64_t x) {
    const uint64_t L = (1ull << 31) - 1;
    x = (x & L) + (x >> 31);
    x = (x & L) + (x >> 31);
    return x >= L ? x - L : x;
}
template <int P> struct mers;
template <> struct mers<31> {
    static constexpr uint64_t L = (1ull << 31) - 1;
    __device__ static uint64_t mul(uint64_t a, uint64_t b) { return mred31(a * b); }
};
template <> struct mers<61> {
    static constexpr uint64_t L = (1ull << 61) - 1;
    __device__ static uint64_t mul(uint64_t a, uint64_t b) { return mred61((unsigned __int128)a * b); }
};

__device__ __forceinline__ uint64_t to_mod(long long v, uint64_t L) {
    long long r = v % (long long)L;
    return (uint64_t)(r < 0 ? r + (long long)L : r);
}

// true iff gcd(p, p') over F_L is a nonzero constant
template <int P>
__device__ bool coprime_mod(const int64_t* c, int d, uint64_t* a, uint64_t* b, int* s_deg) {
    using F = mers<P>;
    const uint64_t L = F::L;
    const int t = threadIdx.x;
    for (int k = t; k <= DMAX; k += blockDim.x) {
        a[k] = k <= d ? to_mod(c[k], L) : 0;
        b[k] = (k + 1 <= d) ? F::mul(to_mod(c[k + 1], L), (uint64_t)(k + 1) % L) : 0;
    }
    __syncthreads();
    if (t == 0) {
        int da = d, db = d - 1;
        while (da >= 0 && a[da] == 0) --da;
        while (db >= 0 && b[db] == 0) --db;
        s_deg[0] = da; s_deg[1] = db;
    }
    __syncthreads();
    int da = s_deg[0], db = s_deg[1];
    bool swapped = false;
    uint64_t* A = a;
    uint64_t* B = b;
    while (db > 0) {
        // A <- A mod B by pseudo-division; every thread then finds the new degree
        // itself (the leading term is cancelled, and lower ones vanish only by
        // chance), so a step takes two barriers
        while (da >= db) {
            const uint64_t la = A[da], lb = B[db];
            const int sh = da - db;
            uint64_t v = 0;
            const int k = t;
            if (k <= da) {
                v = F::mul(lb, A[k]);
                if (k >= sh && k - sh <= db) {
                    v += L - F::mul(la, B[k - sh]);          // both terms below L: one subtraction reduces
                    if (v >= L) v -= L;
                }
            }
            __syncthreads();
            if (k <= da) A[k] = v;
            __syncthreads();
            int nd = da - 1;
            while (nd >= 0 && A[nd] == 0) --nd;
            da = nd;
        }
        // swap roles
        uint64_t* T = A; A = B; B = T;
        int td = da; da = db; db = td;
        swapped = !swapped;
        __syncthreads();
    }
    (void)swapped;
    return db == 0;        // remainder sequence ended in a nonzero constant
}

__global__ void __launch_bounds__(DMAX + 1)
k_validate(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
           int32_t* __restrict__ status) {
    __shared__ uint64_t a[DMAX + 1], b[DMAX + 1];
    __shared__ int s_deg[2], s_bad;
    const int prob = blockIdx.x, t = threadIdx.x;
    const int d = degrees[prob];
    const int64_t* c = coeffs + (size_t)prob * LDC;
    if (d < 1 || d > DMAX) { if (t == 0) status[prob] = RFR_E_RANGE; return; }
    if (t == 0) s_bad = 0;
    __syncthreads();
    if (t <= d) {
        const long long v = c[t];
        if (v >= (1ll << 53) || v <= -(1ll << 53)) atomicExch(&s_bad, RFR_E_RANGE);
    }
    __syncthreads();
    if (s_bad) { if (t == 0) status[prob] = s_bad; return; }
    if (c[d] != 1) { if (t == 0) status[prob] = RFR_E_NOT_MONIC; return; }
    if (d == 1) { if (t == 0) status[prob] = RFR_OK; return; }
    bool ok = coprime_mod<31>(c, d, a, b, s_deg);
    __syncthreads();
    if (!ok) ok = coprime_mod<61>(c, d, a, b, s_deg);
    if (t == 0) status[prob] = ok ? RFR_OK : RFR_SF_SUSPECT;
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_validate(const int64_t* coeffs, const int32_t* degrees, int batch,
                                  int32_t* status, void* stream) {
    if (batch < 0 || !coeffs || !degrees || !status) return RFR_E_INVALID;
    if (batch == 0) return RFR_OK;
    k_validate<<<batch, DMAX + 1, 0, (cudaStream_t)stream>>>(coeffs, degrees, status);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
