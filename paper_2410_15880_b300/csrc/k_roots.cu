// k_roots.cu — K-a: batched root finder (the "black box" of Section 2).
//
// Three kernels: k_aberth (one CTA per polynomial, one thread per root,
// d <= 128) for steps 1-2; k_polish and k_radius (one warp per 32 roots,
// spread over the whole GPU, because the double-double work is FP64-bound and
// independent per root) for steps 3 and 4.
//  1. Starting points from the Newton polygon of p (upper convex hull of
//     (k, log|a_k|)): for each hull edge of width m, m points on a circle
//     whose radius is the edge's geometric-mean root modulus (Bini 1996).
//  2. Aberth-Ehrlich iteration (Jacobi form):
//        z_i <- z_i - N_i / (1 - N_i * sum_{j != i} 1/(z_i - z_j)),
//     N_i = p(z_i)/p'(z_i).  For |z| > 1 the reversed polynomial
//     P(w) = w^d p(1/w) is evaluated at w = 1/z, so nothing overflows:
//        p/p' = z P(w) / (d P(w) - w P'(w)).
//     A root stops moving when its correction is below 4 ulp or |p(z_i)| is
//     below the rounding-error bound of its evaluation.  In FP32-bulk mode
//     the same iteration runs in FP32 first and FP64 finishes it.
//  3. One Newton step with p evaluated in double-double arithmetic (the
//     correction itself in FP64), so each root is kept as a DD value.
//  4. Inclusion radius: r_i = d |p(z_i)| / prod_{j != i} |z_i - z_j|, with
//     |p(z_i)| enlarged by the DD evaluation's error bound.  When the discs
//     D(z_i, r_i) are pairwise disjoint each holds exactly one root of p
//     (the Weierstrass / Braess-Hadeler inclusion theorem).
#include "rfr_device.cuh"

namespace rfr {

template <typename T> struct cx { T x, y; };
template <typename T> __device__ __forceinline__ cx<T> cxm(T x, T y) { return {x, y}; }
template <typename T> __device__ __forceinline__ cx<T> operator+(cx<T> a, cx<T> b) { return {a.x + b.x, a.y + b.y}; }
template <typename T> __device__ __forceinline__ cx<T> operator-(cx<T> a, cx<T> b) { return {a.x - b.x, a.y - b.y}; }
template <typename T> __device__ __forceinline__ cx<T> operator*(cx<T> a, cx<T> b) {
    return {a.x * b.x - a.y * b.y, a.x * b.y + a.y * b.x};
}
template <typename T> __device__ __forceinline__ cx<T> cscale(cx<T> a, T s) { return {a.x * s, a.y * s}; }
template <typename T> __device__ __forceinline__ T cabs2(cx<T> a) { return a.x * a.x + a.y * a.y; }
template <typename T> __device__ __forceinline__ T cabsv(cx<T> a);
template <> __device__ __forceinline__ double cabsv(cx<double> a) { return hypot(a.x, a.y); }
template <> __device__ __forceinline__ float cabsv(cx<float> a) { return hypotf(a.x, a.y); }
template <typename T> __device__ __forceinline__ cx<T> cdivv(cx<T> a, cx<T> b) {
    T s = fmax(fabs(b.x), fabs(b.y));
    if (s == T(0)) return {T(0), T(0)};
    T bx = b.x / s, by = b.y / s;
    T m = (bx * bx + by * by) * s;
    return {(a.x * bx + a.y * by) / m, (a.y * bx - a.x * by) / m};
}
template <typename T> struct eps_of;
template <> struct eps_of<double> { static constexpr double v = 1.1102230246251565e-16; };
template <> struct eps_of<float> { static constexpr float v = 5.9604645e-8f; };

// Newton ratio p(z)/p'(z); *noise = |p(z)| is below its evaluation error bound.
template <typename T>
__device__ cx<T> newton_ratio(const T* a, int d, cx<T> z, bool* noise) {
    T az = cabsv(z);
    const T g = T(4 * (2 * d + 2)) * eps_of<T>::v;
    if (az <= T(1)) {
        cx<T> p = cxm<T>(a[d], 0), dp = cxm<T>(0, 0);
        T mag = fabs(a[d]);
        for (int k = d - 1; k >= 0; --k) {
            dp = dp * z + p;
            p = p * z + cxm<T>(a[k], 0);
            mag = mag * az + fabs(a[k]);
        }
        *noise = cabsv(p) <= g * mag;
        return cdivv(p, dp);
    }
    cx<T> w = cdivv(cxm<T>(1, 0), z);
    T aw = cabsv(w);
    cx<T> P = cxm<T>(a[0], 0), dP = cxm<T>(0, 0);
    T mag = fabs(a[0]);
    for (int k = 1; k <= d; ++k) {
        dP = dP * w + P;
        P = P * w + cxm<T>(a[k], 0);
        mag = mag * aw + fabs(a[k]);
    }
    *noise = cabsv(P) <= g * mag;
    cx<T> den = cscale(P, T(d)) - w * dP;
    return cdivv(z * P, den);
}

// Aberth iterations on the shared approximations z[0..d); returns true when
// every root stopped moving.
template <typename T>
__device__ bool aberth(const T* a, int d, cx<T>* z, int max_iter, int* s_flag) {
    const int i = threadIdx.x;
    bool done = i >= d;
    for (int it = 0; it < max_iter; ++it) {
        cx<T> zi = i < d ? z[i] : cxm<T>(0, 0);
        cx<T> corr = cxm<T>(0, 0);
        if (!done) {
            bool noise;
            cx<T> N = newton_ratio<T>(a, d, zi, &noise);
            // The Aberth sum sum_j 1/(z_i - z_j) only steers the step (near
            // convergence N S << 1 damps its error), so it is accumulated in
            // FP32 from differences taken in T; the Newton ratio N keeps T.
            float sx = 0.f, sy = 0.f;
            for (int j = 0; j < d; ++j) {
                if (j == i) continue;
                const float dx = (float)(zi.x - z[j].x), dy = (float)(zi.y - z[j].y);
                const float m = dx * dx + dy * dy;
                if (m > 0.f) {
                    const float r = 1.f / m;
                    sx += dx * r;
                    sy -= dy * r;
                }
            }
            const cx<T> S = cxm<T>((T)sx, (T)sy);
            cx<T> den = cxm<T>(1, 0) - N * S;
            corr = cdivv(N, den);
            if (!(cabsv(corr) < T(1e30))) corr = N;               // degenerate denominator: Newton step
            if (noise || cabsv(corr) <= T(4) * eps_of<T>::v * cabsv(zi)) done = true;
        }
        __syncthreads();
        if (i < d) z[i] = zi - corr;
        if (!__syncthreads_or(!done)) return true;
    }
    return false;
}

// p(Z) in double-double (|z| <= 1) or P(W), W = 1/Z (|z| > 1).
__device__ cdd eval_dd(const double* a, int d, cdd Z, bool reversed) {
    if (!reversed) {
        cdd P = cdd_make(a[d], 0.0);
        for (int k = d - 1; k >= 0; --k) P = cdd_add_d(cdd_mul(P, Z), a[k]);
        return P;
    }
    cdd P = cdd_make(a[0], 0.0);
    for (int k = 1; k <= d; ++k) P = cdd_add_d(cdd_mul(P, Z), a[k]);
    return P;
}

// Kernel 1: Aberth iterations, one CTA per polynomial.  Writes the FP64
// approximations to roots[.., 0] / roots[.., 2] and the convergence status.
__global__ void __launch_bounds__(DMAX)
k_aberth(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
         int root_mode, double* __restrict__ roots, int32_t* __restrict__ status) {
    __shared__ double a[DMAX + 1];
    __shared__ float af[DMAX + 1];
    __shared__ cx<double> z[DMAX];
    __shared__ cx<float> zf[DMAX];
    __shared__ int hull[DMAX + 2];
    __shared__ int nhull, kmin, s_flag;

    const int prob = blockIdx.x, i = threadIdx.x;
    const int d = degrees[prob];
    const int64_t* c = coeffs + (size_t)prob * LDC;
    const int pre = status[prob];
    if (pre < 0) return;                       // rejected by the input checks
    if (d < 1 || d > DMAX) {
        if (i == 0) status[prob] = RFR_E_RANGE;
        return;
    }
    for (int k = i; k <= d; k += blockDim.x) { a[k] = (double)c[k]; af[k] = (float)c[k]; }
    __syncthreads();

    // Newton polygon: upper hull of (k, log2|a_k|) over a_k != 0.
    if (i == 0) {
        int km = 0;
        while (km < d && a[km] == 0.0) ++km;
        kmin = km;
        int h = 0;
        for (int k = km; k <= d; ++k) {
            if (a[k] == 0.0) continue;
            double yk = log2(fabs(a[k]));
            while (h >= 2) {
                int o = hull[h - 2], p = hull[h - 1];
                double yo = log2(fabs(a[o])), yp = log2(fabs(a[p]));
                double cr = (double)(p - o) * (yk - yo) - (yp - yo) * (double)(k - o);
                if (cr >= 0.0) --h; else break;
            }
            hull[h++] = k;
        }
        nhull = h;
    }
    __syncthreads();
    if (i < d) {
        cx<double> z0 = cxm<double>(0.0, 0.0);
        if (i >= kmin) {
            int e = 0;
            while (e + 1 < nhull - 1 && hull[e + 1] <= i) ++e;
            int k0 = hull[e], k1 = hull[e + 1], m = k1 - k0, j = i - k0;
            double u = exp2((log2(fabs(a[k0])) - log2(fabs(a[k1]))) / (double)m);
            double s, co;
            sincospi(2.0 * ((double)j + 0.25) / (double)m + 0.22 * (double)e + 0.13, &s, &co);
            z0 = cxm<double>(u * co, u * s);
        }
        z[i] = z0;
        zf[i] = cxm<float>((float)z0.x, (float)z0.y);
    }
    __syncthreads();

    bool conv;
    if (root_mode == RFR_ROOTS_FP32_BULK) {
        aberth<float>(af, d, zf, 400, &s_flag);
        if (i < d) z[i] = cxm<double>((double)zf[i].x, (double)zf[i].y);
        __syncthreads();
        conv = aberth<double>(a, d, z, 200, &s_flag);
    } else {
        conv = aberth<double>(a, d, z, 600, &s_flag);
    }
    if (i < d) {
        double* out = roots + ((size_t)prob * DMAX + i) * 4;
        out[0] = z[i].x; out[1] = 0.0; out[2] = z[i].y; out[3] = 0.0;
    }
    if (i == 0) {
        const bool suspect = pre == RFR_SF_SUSPECT;
        status[prob] = conv ? (suspect ? RFR_SF_SUSPECT : RFR_OK)
                            : (suspect ? RFR_E_NOT_SQUAREFREE : RFR_E_NO_CONVERGENCE);
    }
}

// One warp per 32 roots of one polynomial: blockIdx.x = problem * 4 + chunk.
constexpr int CHUNKS = DMAX / 32;
struct RootSlot { int prob, d, i, chunk; };
__device__ __forceinline__ bool root_slot(const int32_t* degrees, const int32_t* status, RootSlot* r) {
    r->prob = blockIdx.x / CHUNKS;
    r->chunk = blockIdx.x % CHUNKS;
    r->d = degrees[r->prob];
    r->i = r->chunk * 32 + threadIdx.x;
    const int st = status[r->prob];
    return (st == RFR_OK || st == RFR_SF_SUSPECT) && r->d >= 1 && r->d <= DMAX;
}

// Kernel 2: one Newton step per root with p evaluated in double-double (the
// correction itself in FP64), so each root becomes a DD value.
__global__ void __launch_bounds__(32)
k_polish(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
         const int32_t* __restrict__ status, double* __restrict__ roots) {
    __shared__ double a[DMAX + 1];
    RootSlot R;
    if (!root_slot(degrees, status, &R)) return;
    const int d = R.d, i = R.i;
    if (R.chunk * 32 >= d) return;
    const int64_t* c = coeffs + (size_t)R.prob * LDC;
    for (int k = threadIdx.x; k <= d; k += 32) a[k] = (double)c[k];
    __syncwarp();
    if (i >= d) return;
    double* out = roots + ((size_t)R.prob * DMAX + i) * 4;
    cdd Z = cdd_make(out[0], out[2]);
    // one Newton step from the FP64 Aberth root (error ~1e-16 |z|) squares the
    // error; the inclusion radius computed afterwards certifies what it reached
    for (int it = 0; it < 1; ++it) {
        cx<double> zh = cxm<double>(Z.re.hi, Z.im.hi);
        bool rev = cabsv(zh) > 1.0;
        cx<double> N;
        if (!rev) {
            cdd P = eval_dd(a, d, Z, false);
            cx<double> p = cxm<double>(a[d], 0), dp = cxm<double>(0, 0);
            for (int k = d - 1; k >= 0; --k) { dp = dp * zh + p; p = p * zh + cxm<double>(a[k], 0); }
            N = cdivv(cxm<double>(P.re.hi, P.im.hi), dp);
        } else {
            cdd W = cdd_inv(Z);
            cdd P = eval_dd(a, d, W, true);
            cx<double> wh = cxm<double>(W.re.hi, W.im.hi);
            cx<double> Pp = cxm<double>(a[0], 0), dP = cxm<double>(0, 0);
            for (int k = 1; k <= d; ++k) { dP = dP * wh + Pp; Pp = Pp * wh + cxm<double>(a[k], 0); }
            cx<double> Ph = cxm<double>(P.re.hi, P.im.hi);
            N = cdivv(zh * Ph, cscale(Ph, (double)d) - wh * dP);
        }
        if (!(cabsv(N) < 1e300)) {                              // degenerate: plain FP64 Newton ratio
            bool noise;
            N = newton_ratio<double>(a, d, zh, &noise);
        }
        Z.re = dd_add_d(Z.re, -N.x);
        Z.im = dd_add_d(Z.im, -N.y);
    }
    out[0] = Z.re.hi; out[1] = Z.re.lo; out[2] = Z.im.hi; out[3] = Z.im.lo;
}

// Kernel 3: inclusion radius r_i = d |p(z_i)| / prod_{j != i} |z_i - z_j| with
// |p(z_i)| from a double-double evaluation plus its error bound.
__global__ void __launch_bounds__(32)
k_radius(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
         const int32_t* __restrict__ status, const double* __restrict__ roots,
         double* __restrict__ radius) {
    __shared__ double a[DMAX + 1];
    __shared__ cx<double> z[DMAX];
    RootSlot R;
    if (!root_slot(degrees, status, &R)) return;
    const int d = R.d, i = R.i;
    if (R.chunk * 32 >= d) return;
    const int64_t* c = coeffs + (size_t)R.prob * LDC;
    const double* Rt = roots + (size_t)R.prob * DMAX * 4;
    for (int k = threadIdx.x; k <= d; k += 32) a[k] = (double)c[k];
    for (int k = threadIdx.x; k < d; k += 32) z[k] = cxm<double>(Rt[4 * k], Rt[4 * k + 2]);
    __syncwarp();
    if (i >= d) return;
    const cdd Z = {{Rt[4 * i], Rt[4 * i + 1]}, {Rt[4 * i + 2], Rt[4 * i + 3]}};
    const cx<double> zh = z[i];
    const double az = cabsv(zh);
    const bool rev = az > 1.0;
    double lp;
    if (!rev) {
        cdd P = eval_dd(a, d, Z, false);
        double mag = 0.0;
        for (int k = d; k >= 0; --k) mag = mag * az + fabs(a[k]);
        double pv = hypot(P.re.hi, P.im.hi);
        double err = (double)(2 * d + 8) * 0x1p-100 * mag;
        lp = log2(pv + err);
    } else {
        cdd W = cdd_inv(Z);
        cdd P = eval_dd(a, d, W, true);
        double aw = 1.0 / az, mag = 0.0;
        for (int k = 0; k <= d; ++k) mag = mag * aw + fabs(a[k]);
        double pv = hypot(P.re.hi, P.im.hi);
        double err = (double)(2 * d + 8) * 0x1p-100 * mag;
        lp = (double)d * log2(az) + log2(pv + err);
    }
    // log2 of prod_{j != i} |z_i - z_j| in FP32 (d <= 128 terms, each with
    // relative error ~1e-7: the sum is within 2e-5 of the exact value,
    // far inside the 1.01 safety factor below)
    float lprodf = 0.f;
    bool coincide = false;
    for (int j = 0; j < d; ++j) {
        if (j == i) continue;
        const float dist = (float)cabsv(zh - z[j]);
        if (!(dist > 0.f)) coincide = true; else lprodf += log2f(dist);
    }
    const double lprod = (double)lprodf;
    double r = coincide ? INFINITY : exp2(log2((double)d) + lp - lprod) * 1.01 + 0x1p-96 * az;
    if (d == 1) r = 0x1p-96 * az + 0x1p-100;
    radius[(size_t)R.prob * DMAX + i] = r;
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_roots(const int64_t* coeffs, const int32_t* degrees, int batch,
                               int root_mode, double* roots, double* radius,
                               int32_t* status, void* stream) {
    if (batch < 0 || !coeffs || !degrees || !roots || !radius || !status) return RFR_E_INVALID;
    if (batch == 0) return RFR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_aberth<<<batch, DMAX, 0, s>>>(coeffs, degrees, root_mode, roots, status);
    k_polish<<<batch * CHUNKS, 32, 0, s>>>(coeffs, degrees, status, roots);
    k_radius<<<batch * CHUNKS, 32, 0, s>>>(coeffs, degrees, status, roots, radius);
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
