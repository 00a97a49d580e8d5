// k_verify.cu — K-f: the candidate test of Algorithm FACTOR (Section 2).
//
// One warp per job (a problem and a pattern over its n elements).  The real
// factor of Eq. 2 for the pattern, or for its complement when that has the
// lower degree (so the built factor has degree e <= d/2), is multiplied out
// in double-double arithmetic from the DD roots: one linear factor x - u or
// one quadratic x^2 - (z + z')x + z z' per element; lane l owns coefficients
// l, l+32, l+64.  Each coefficient must lie within 1/4 of an integer, and
// within 2^20 times the bound that the inclusion radii put on its error,
// and below 2^62 in magnitude, otherwise the pattern is rejected.  The rounded
// monic q then divides p exactly: long division in 128-bit integers, each
// quotient coefficient required below 2^62 in magnitude, and the remainder
// must vanish.  Only this exact step decides acceptance.
#include "rfr_device.cuh"

namespace rfr {

constexpr int QMAX = DMAX / 2 + 1;    // coefficients of a factor of degree <= 64

__device__ __forceinline__ bool patbit(uint64_t lo, uint64_t hi, int k) {
    return k < 64 ? ((lo >> k) & 1ull) : ((hi >> (k - 64)) & 1ull);
}

// VW warps (jobs) per CTA.  A job is bound by the FP64 pipe of its SM (a warp's
// FP64 instruction occupies it for many cycles on this GPU), so a small batch
// of jobs runs one warp per CTA, spread over the SMs.
template <int VW>
__global__ void __launch_bounds__(VW * 32)
k_verify(const int64_t* __restrict__ coeffs, const double* __restrict__ roots,
         const rfr_plan* __restrict__ plans, const int32_t* __restrict__ prob,
         const uint64_t* __restrict__ pat_lo, const uint64_t* __restrict__ pat_hi, int jobs,
         int32_t* __restrict__ result, int64_t* __restrict__ coeffs_out) {
    __shared__ dd qs[VW][QMAX + 1];
    __shared__ long long qi[VW][QMAX + 1];
    __shared__ __int128 rs[VW][DMAX + 1];
    __shared__ long long quo[VW][DMAX + 1];
    __shared__ dd cA[VW][DMAX], cB[VW][DMAX];     // per element of the built side: u, or z + z' and Re(z z')
    __shared__ signed char ek[VW][DMAX];          // 0: not in the built side, else its kind (1 or 2)
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int job = blockIdx.x * VW + w;
    if (job >= jobs) return;
    const int pi = prob[job];
    const rfr_plan& P = plans[pi];
    const uint64_t lo = pat_lo[job], hi = pat_hi[job];
    if (P.status != RFR_OK || P.n < 1) {
        if (lane == 0) result[job] = P.status != RFR_OK ? P.status : RFR_E_INVALID;
        return;
    }
    const int n = P.n, d = P.degree;
    int degP = 0;
    for (int k = lane; k < n; k += 32) degP += patbit(lo, hi, k) ? P.kind[k] : 0;
    for (int o = 16; o; o >>= 1) degP += __shfl_xor_sync(0xffffffffu, degP, o);
    const bool comp = degP > d - degP;
    const int e = comp ? d - degP : degP;
    const double* R = roots + (size_t)pi * DMAX * 4;

    // ---- multiply out the chosen side in double-double
    for (int j = lane; j <= QMAX; j += 32) qs[w][j] = dd_make(j == 0 ? 1.0 : 0.0);
    __syncwarp();
    // Integrality tolerance.  Moving each root z_k by at most the inclusion
    // radius r moves every coefficient of q = prod (x - z_k) by at most
    // B = prod_k (1 + |z_k| + r) - prod_k (1 + |z_k|) <= r * PA * sum_k 1 / (1 + |z_k| + r)
    // with PA = prod_k (1 + |z_k| + r); the double-double products add about
    // PA * 2^-90.  A coefficient must lie within 2^20 times that of an integer
    // (and within 1/4): with only the 1/4 test, a pattern that is not a
    // divisor but whose coefficients all fall near integers by chance rounds
    // to some other divisor of p, passes the exact division, and ties the
    // wrong roots to that divisor.
    const double rr = P.max_radius;
    double pa = 1.0, sinv = 0.0;
    auto acc = [&](double m) { const double a = 1.0 + m + rr; pa *= a; sinv += 1.0 / a; };
    // The built side's factors, read from the plan and the roots by all lanes at
    // once into shared memory (the product below walks them in order).
    for (int k = lane; k < n; k += 32) {
        const bool in = patbit(lo, hi, k) != comp;
        const int kind = in ? P.kind[k] : 0;
        if (in) {
            const double* r0 = R + 4 * P.root0[k];
            if (kind == 1) {
                cA[w][k] = {r0[0], r0[1]};
                acc(fabs(r0[0]));
            } else {
                const double* r1 = R + 4 * P.root1[k];
                const dd x0 = {r0[0], r0[1]}, y0 = {r0[2], r0[3]};
                const dd x1 = {r1[0], r1[1]}, y1 = {r1[2], r1[3]};
                cA[w][k] = dd_add(x0, x1);                                 // z + z'
                cB[w][k] = dd_sub(dd_mul(x0, x1), dd_mul(y0, y1));         // Re(z z')
                acc(hypot(r0[0], r0[2]));
                acc(hypot(r1[0], r1[2]));
            }
        }
        ek[w][k] = (signed char)kind;
    }
    for (int o = 16; o; o >>= 1) {
        pa *= __shfl_xor_sync(0xffffffffu, pa, o);
        sinv += __shfl_xor_sync(0xffffffffu, sinv, o);
    }
    __syncwarp();
    int cur = 0;
    for (int k = 0; k < n; ++k) {
        const int kind = ek[w][k];
        if (!kind) continue;
        // slots of 32 coefficients that the product reaches after this step (warp-uniform):
        // the others are skipped whole, which saves their FP64 work
        const int ns = min(3, (cur + 2) / 32 + 1);
        dd old[3], prev[3], prev2[3];
#pragma unroll
        for (int t = 0; t < 3; ++t) {
            if (t >= ns) break;
            const int j = lane + 32 * t;
            old[t] = (j <= QMAX) ? qs[w][j] : dd_make(0.0);
            prev[t] = (j >= 1 && j - 1 <= QMAX) ? qs[w][j - 1] : dd_make(0.0);
            prev2[t] = (j >= 2 && j - 2 <= QMAX) ? qs[w][j - 2] : dd_make(0.0);
        }
        __syncwarp();
        if (kind == 1) {
            const dd u = cA[w][k];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t >= ns) break;
                const int j = lane + 32 * t;
                if (j <= cur + 1 && j <= QMAX) qs[w][j] = dd_sub(prev[t], dd_mul(u, old[t]));
            }
            cur += 1;
        } else {
            const dd tt = cA[w][k], mm = cB[w][k];
#pragma unroll
            for (int t = 0; t < 3; ++t) {
                if (t >= ns) break;
                const int j = lane + 32 * t;
                if (j <= cur + 2 && j <= QMAX)
                    qs[w][j] = dd_add(dd_sub(prev2[t], dd_mul(tt, prev[t])), dd_mul(mm, old[t]));
            }
            cur += 2;
        }
        __syncwarp();
    }

    // ---- round and test integrality
    bool ok = true;
    const double tol = fmin(0.25, 0x1p20 * (rr * pa * sinv + pa * 0x1p-90));
    for (int j = lane; j <= e; j += 32) {
        const dd v = qs[w][j];
        const double r = rint(v.hi);
        const double f = (v.hi - r) + v.lo;
        if (!(fabs(f) < tol) || !(fabs(r) < 0x1p62)) ok = false;
        else qi[w][j] = (long long)r;
    }
    ok = __all_sync(0xffffffffu, ok);
    __syncwarp();
    if (ok && qi[w][e] != 1) ok = false;
    if (!ok) {
        if (lane == 0) result[job] = 0;
        return;
    }

    // ---- exact division p / q in 128-bit integers
    const int64_t* pc = coeffs + (size_t)pi * LDC;
    for (int j = lane; j <= d; j += 32) rs[w][j] = (__int128)pc[j];
    __syncwarp();
    bool ovf = false;
    const __int128 lim = (__int128)1 << 125;
    for (int k = d - e; k >= 0; --k) {
        const __int128 h = rs[w][k + e];
        if (h >= ((__int128)1 << 62) || h <= -((__int128)1 << 62)) { ovf = true; break; }
        if (lane == 0) quo[w][k] = (long long)h;
        for (int j = lane; j < e; j += 32) {
            __int128 v = rs[w][k + j] - h * (__int128)qi[w][j];
            if (v > lim || v < -lim) ovf = true;
            rs[w][k + j] = v;
        }
        ovf = __any_sync(0xffffffffu, ovf);
        __syncwarp();
        if (ovf) break;
    }
    bool zero = true;
    if (!ovf)
        for (int j = lane; j < e; j += 32) zero = zero && rs[w][j] == 0;
    zero = __all_sync(0xffffffffu, zero);
    int res;
    if (ovf) res = RFR_E_OVERFLOW;
    else res = zero ? 1 : 0;
    if (lane == 0) result[job] = res;
    if (res == 1 && coeffs_out) {
        int64_t* out = coeffs_out + (size_t)job * LDC;
        if (!comp) {
            for (int j = lane; j <= e; j += 32) out[j] = qi[w][j];
        } else {
            for (int j = lane; j <= d - e; j += 32) out[j] = quo[w][j];
        }
    }
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_verify(const int64_t* coeffs, const int32_t* degrees,
                                const double* roots, const rfr_plan* plans,
                                const int32_t* prob, const uint64_t* pat_lo,
                                const uint64_t* pat_hi, int jobs,
                                int32_t* result, int64_t* coeffs_out, void* stream) {
    (void)degrees;
    if (jobs < 0 || !coeffs || !roots || !plans || !prob || !pat_lo || !pat_hi || !result) return RFR_E_INVALID;
    if (jobs == 0) return RFR_OK;
    if (jobs <= 4 * 148)
        k_verify<1><<<jobs, 32, 0, (cudaStream_t)stream>>>(coeffs, roots, plans, prob, pat_lo, pat_hi, jobs, result, coeffs_out);
    else
        k_verify<4><<<(jobs + 3) / 4, 128, 0, (cudaStream_t)stream>>>(coeffs, roots, plans, prob, pat_lo, pat_hi, jobs, result, coeffs_out);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
