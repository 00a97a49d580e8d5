// k_weights.cu — K-b: real factorisation (Eq. 1) and fixed-point weights.
//
// One CTA per polynomial, one thread per root.
//  * Disjointness: every pair of inclusion discs must be disjoint, else the
//    roots are not separated (RFR_E_ROOTS).
//  * Real or not: a root whose disc misses the real axis (|Im z| > r) is not
//    real.  A root with |Im z| <= r is real when no other disc comes within
//    3r of it: the conjugate of its root lies within 3r of z, hence in the
//    same disc, which holds only one root.  Anything else is undecidable
//    (RFR_E_ROOTS).
//  * Each root with Im z > 0 is paired with the Im z < 0 root nearest its
//    conjugate; the pairing must be a bijection and the partner disc must
//    meet the conjugate disc.
//  * Elements in canonical order: real roots ascending, then pairs by
//    (Re z, Im z).  Tr_1 part t1 = u or Re z + Re z' (Eq. 4), Tr_2 part
//    t2 = u^2 or Re z^2 + Re z'^2, both in double-double; each is scaled to
//    w = round(frac(t) * 2^64) mod 2^64, i.e. Eq. 18 with M = 2^64 and
//    rounding in place of floor.
//  * Windows: a subset sum of the w's differs from 2^64 x (the true Tr_1 of
//    that subset) by at most 2^64 * sum_k err_k + n/2, with err_k the
//    element's radius (or the two radii of a pair); W adds slack to that.
//    W2 is the same bound for Tr_2, err2 = (2|z| + r) r per root.
#include "rfr_device.cuh"

namespace rfr {

// An unsigned key with the order of the finite double x (-0 and +0 equal), so
// the canonical order is taken with integer compares instead of FP64 ones.
__device__ __forceinline__ unsigned long long order_key(double x) {
    const unsigned long long u = (unsigned long long)__double_as_longlong(x + 0.0);   // -0 + 0 = +0
    return (u >> 63) ? ~u : (u | 0x8000000000000000ull);
}

__global__ void __launch_bounds__(DMAX)
k_weights(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees, const double* __restrict__ roots,
          const double* __restrict__ radius, const int32_t* __restrict__ root_status,
          double eps_override, rfr_plan* __restrict__ plans) {
    __shared__ double zx[DMAX], zy[DMAX], rr[DMAX];
    __shared__ float zxf[DMAX], zyf[DMAX], rrf[DMAX], azf[DMAX];   // FP32 copies for the disc prefilter
    __shared__ unsigned long long kx[DMAX], ky[DMAX];              // order-preserving keys of Re z, Im z
    __shared__ int cls[DMAX];        // 0 real, 1 upper, 2 lower
    __shared__ int partner[DMAX], taken[DMAX];
    __shared__ int s_err, s_r, s_c;
    __shared__ double s_e1, s_e2, s_maxr, s_res;
    const int prob = blockIdx.x, i = threadIdx.x;
    const int d = degrees[prob];
    rfr_plan* P = plans + prob;
    const int rs = root_status[prob];
    const bool suspect = rs == RFR_SF_SUSPECT;
    const int fail = suspect ? RFR_E_NOT_SQUAREFREE : RFR_E_ROOTS;
    if ((rs != RFR_OK && !suspect) || d < 1 || d > DMAX) {
        if (i == 0) {
            P->status = rs != RFR_OK ? rs : RFR_E_RANGE;
            P->degree = d;
            P->n = P->r = P->c = P->n_a = P->n_b = 0;
        }
        return;
    }
    const double* R = roots + (size_t)prob * DMAX * 4;
    if (i < d) {
        zx[i] = R[4 * i];
        zy[i] = R[4 * i + 2];
        rr[i] = radius[(size_t)prob * DMAX + i];
        taken[i] = 0;
        partner[i] = -1;
        zxf[i] = (float)zx[i];
        zyf[i] = (float)zy[i];
        azf[i] = fmaxf(fabsf(zxf[i]), fabsf(zyf[i]));
        // the radius rounded up (infinite or NaN radii stay so: they fail the prefilter)
        const float rf = (float)rr[i];
        rrf[i] = rf * (1.f + 0x1p-20f) + 0x1p-149f;
        kx[i] = order_key(zx[i]);
        ky[i] = order_key(zy[i]);
    }
    if (i == 0) { s_err = 0; s_r = 0; s_c = 0; s_e1 = 0.0; s_e2 = 0.0; s_maxr = 0.0; s_res = 0.0; }
    __syncthreads();
    if (i < d) {
        // FP64 relative residual |p(z)| / sum |a_k| |z|^k of the root's FP64 part
        // (reversed polynomial at 1/z when |z| > 1, where the ratio is the same)
        const int64_t* c = coeffs + (size_t)prob * LDC;
        const double az = hypot(zx[i], zy[i]);
        double pr, pi, mag;
        if (az <= 1.0) {
            pr = (double)c[d]; pi = 0.0; mag = fabs(pr);
            for (int k = d - 1; k >= 0; --k) {
                const double t = pr * zx[i] - pi * zy[i] + (double)c[k];
                pi = pr * zy[i] + pi * zx[i];
                pr = t;
                mag = mag * az + fabs((double)c[k]);
            }
        } else {
            const double wx = zx[i] / (az * az), wy = -zy[i] / (az * az), aw = 1.0 / az;
            pr = (double)c[0]; pi = 0.0; mag = fabs(pr);
            for (int k = 1; k <= d; ++k) {
                const double t = pr * wx - pi * wy + (double)c[k];
                pi = pr * wy + pi * wx;
                pr = t;
                mag = mag * aw + fabs((double)c[k]);
            }
        }
        const double res = hypot(pr, pi) / mag;
        atomicMax((unsigned long long*)&s_res, __double_as_longlong(isfinite(res) ? res : 1e308));
    }
    __syncthreads();

    if (i < d) {
        double ri = rr[i];
        bool isolated = isfinite(ri), strong = true;
        // squared distances against squared radius sums (no square roots: FP64
        // is this part's limit; an infinite or NaN radius fails both tests).
        // An FP32 prefilter settles the pairs that are far apart: the FP32
        // difference of the FP32 copies is within 2^-22 (|z_i| + |z_j|) (max
        // norm) of the exact one, so when |f|^2 exceeds (s3 + that)^2 with a
        // 2^-20 margin, the roots are certainly more than s3 >= s1 apart and
        // both tests pass; only near pairs take the FP64 test.
        const float rif = rrf[i], azi = azf[i], zxi = zxf[i], zyi = zyf[i];
        for (int j = 0; j < d; ++j) {
            if (j == i) continue;
            const float fx = zxi - zxf[j], fy = zyi - zyf[j];
            const float d2f = fx * fx + fy * fy;
            const float b = 3.f * rif + rrf[j] + 0x1p-22f * (azi + azf[j]);
            if (d2f > b * b * (1.f + 0x1p-20f)) continue;
            const double dx = zx[i] - zx[j], dy = zy[i] - zy[j];
            const double d2 = dx * dx + dy * dy;
            const double s1 = ri + rr[j], s3 = 3.0 * ri + rr[j];
            if (!(d2 > s1 * s1)) isolated = false;
            if (!(d2 > s3 * s3)) strong = false;
        }
        int k;
        if (!isolated) k = -1;
        else if (fabs(zy[i]) > ri) k = zy[i] > 0.0 ? 1 : 2;
        else k = strong ? 0 : -1;
        cls[i] = k;
        if (k < 0) atomicExch(&s_err, 1);
        atomicMax((unsigned long long*)&s_maxr, __double_as_longlong(isfinite(ri) ? ri : 1e308));
    }
    __syncthreads();
    if (s_err) {
        if (i == 0) { P->status = fail; P->degree = d; P->n = 0; P->max_radius = s_maxr; }
        return;
    }
    if (i < d && cls[i] == 1) {
        int best = -1;
        double bd2 = INFINITY;                    // squared distance to the conjugate
        for (int j = 0; j < d; ++j) {
            if (cls[j] != 2) continue;
            const double dx = zx[j] - zx[i], dy = zy[j] + zy[i];
            const double d2 = dx * dx + dy * dy;
            if (d2 < bd2) { bd2 = d2; best = j; }
        }
        const double sr = best < 0 ? 0.0 : rr[i] + rr[best];
        if (best < 0 || !(bd2 <= sr * sr)) atomicExch(&s_err, 1);
        else { partner[i] = best; atomicAdd(&taken[best], 1); }
    }
    __syncthreads();
    if (i < d && cls[i] == 2 && taken[i] != 1) atomicExch(&s_err, 1);
    if (i < d && cls[i] == 0) atomicAdd(&s_r, 1);
    if (i < d && cls[i] == 1) atomicAdd(&s_c, 1);
    __syncthreads();
    if (s_err || s_r + 2 * s_c != d) {
        if (i == 0) { P->status = fail; P->degree = d; P->n = 0; P->max_radius = s_maxr; }
        return;
    }
    const int r = s_r, c = s_c, n = r + c;

    if (i < d && cls[i] != 2) {
        // canonical position
        int rank = 0;
        for (int j = 0; j < d; ++j) {
            if (j == i || cls[j] != cls[i]) continue;
            bool before = cls[i] == 0
                ? (kx[j] < kx[i] || (kx[j] == kx[i] && j < i))
                : (kx[j] < kx[i] || (kx[j] == kx[i] && (ky[j] < ky[i] || (ky[j] == ky[i] && j < i))));
            rank += before;
        }
        const int k = cls[i] == 0 ? rank : r + rank;
        const double* Ri = R + 4 * i;
        dd re = {Ri[0], Ri[1]}, im = {Ri[2], Ri[3]};
        dd t1, t2;
        double e1, e2;
        if (cls[i] == 0) {
            t1 = re;
            t2 = dd_mul(re, re);
            e1 = rr[i];
            e2 = (2.0 * fabs(re.hi) + rr[i]) * rr[i];
        } else {
            const int j = partner[i];
            const double* Rj = R + 4 * j;
            dd rej = {Rj[0], Rj[1]}, imj = {Rj[2], Rj[3]};
            t1 = dd_add(re, rej);
            t2 = dd_add(dd_sub(dd_mul(re, re), dd_mul(im, im)), dd_sub(dd_mul(rej, rej), dd_mul(imj, imj)));
            e1 = rr[i] + rr[j];
            double azi = hypot(re.hi, im.hi), azj = hypot(rej.hi, imj.hi);
            e2 = (2.0 * azi + rr[i]) * rr[i] + (2.0 * azj + rr[j]) * rr[j];
        }
        e1 += 0x1p-100 * (fabs(t1.hi) + 1.0);
        e2 += 0x1p-98 * (fabs(t2.hi) + 1.0);
        P->w[k] = dd_frac_fixed64(t1);
        P->w2[k] = dd_frac_fixed64(t2);
        P->kind[k] = cls[i] == 0 ? 1 : 2;
        P->root0[k] = (uint8_t)i;
        P->root1[k] = (uint8_t)(cls[i] == 0 ? i : partner[i]);
        atomicAdd(&s_e1, e1);
        atomicAdd(&s_e2, e2);
    }
    __syncthreads();
    if (i == 0) {
        // W = ceil(2^64 * sum err1 * (1 + 2^-20)) + n + 2, saturating at 2^62.
        double w1 = ldexp(s_e1 * (1.0 + 0x1p-20), 64);
        uint64_t W = w1 >= 0x1p62 ? (1ull << 62) : (uint64_t)ceil(w1) + (uint64_t)n + 2ull;
        if (eps_override > 0.0) {
            double wo = ldexp(eps_override, 64);
            W = wo >= 0x1p62 ? (1ull << 62) : (uint64_t)ceil(wo);
        }
        double w2 = ldexp(s_e2 * (1.0 + 0x1p-20), 64);
        uint64_t W2 = w2 >= 0x1p61 ? (1ull << 63) : (uint64_t)ceil(w2) + (uint64_t)n + 2ull;
        P->status = RFR_OK;
        P->degree = d;
        P->n = n; P->r = r; P->c = c;
        P->n_a = (n - 1) / 2;
        P->n_b = (n - 1) - (n - 1) / 2;
        P->window = W;
        P->window2 = W2;
        P->max_radius = s_maxr;
        P->max_rel_residual = s_res;
        P->sum_err1 = s_e1;
        P->sum_err2 = s_e2;
    }
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_weights(const int64_t* coeffs, const int32_t* degrees, int batch,
                                 const double* roots, const double* radius,
                                 const int32_t* root_status, double eps_override,
                                 rfr_plan* plans, void* stream) {
    if (batch < 0 || !coeffs || !degrees || !roots || !radius || !root_status || !plans) return RFR_E_INVALID;
    if (batch == 0) return RFR_OK;
    k_weights<<<batch, DMAX, 0, (cudaStream_t)stream>>>(coeffs, degrees, roots, radius, root_status, eps_override, plans);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
