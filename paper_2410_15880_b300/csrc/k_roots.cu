// k_roots.cu — K-a: batched root finder (the "black box" of Section 2).
//
// Kernels: k_aberth (one CTA per polynomial, SL = 8 lanes per root,
// d <= 128) for steps 1-2 (in FP32-bulk mode only the FP32 iterations and
// the starting points); k_aberth64 (FP32-bulk mode: the FP64 iterations, one
// polynomial per cluster of 4 CTAs); k_polish and k_radius (SL lanes per
// root, the polynomial split over them, spread over the whole GPU) for steps
// 3 and 4.
// Every evaluation of p is a split Horner scheme over the root's SL lanes:
// the dependent chain is about d / SL steps, and a CTA holds SL times the
// warps of one thread per root, so the iteration is not latency-bound.
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
//  3. A Newton step with p evaluated in double-double arithmetic (the
//     correction itself in FP64), so each root is kept as a DD value; a root
//     whose step was not tiny against the distance to its nearest neighbour
//     (close roots) takes up to four more.
//  4. Inclusion radius: r_i = d |p(z_i)| / prod_{j != i} |z_i - z_j|, with
//     |p(z_i)| enlarged by the DD evaluation's error bound.  When the discs
//     D(z_i, r_i) are pairwise disjoint each holds exactly one root of p
//     (the Weierstrass / Braess-Hadeler inclusion theorem).
#include <cooperative_groups.h>
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

constexpr int SL = 8;                         // lanes per root in every kernel of this file

// x^e for e >= 1 by squaring (a chain of about 2 log2 e products, not e - 1)
template <typename V, class Mul>
__device__ __forceinline__ V pow_sq(V x, int e, Mul mul) {
    V r = x;
    bool have = false;
    while (e) {
        if (e & 1) { r = have ? mul(r, x) : x; have = true; }
        e >>= 1;
        if (e) x = mul(x, x);
    }
    return r;
}

// p(x) in T, and p'(x) and sum_k |c(k)| |x|^k in FP32, for the polynomial
// sum_{k=0}^{n} c(k) x^k, split over the root's SL lanes (mask: the lanes of the
// warp taking part, whole roots only).  Lane l of a root takes the
// B = ceil((n+1)/SL) coefficients k in [lB, lB + B) by Horner (three
// independent chains); a shuffle tree adds the lanes' parts times x^(lB).  The
// root's first lane holds the result.  Only p needs T: near a root the Newton
// ratio p / p' keeps the relative accuracy of p' (1e-7 in FP32), so each FP64
// step still shrinks the error by about that factor, and the error bound
// needs no more; FP64 is the slow part of this GPU.
template <typename T> struct Eval3 { cx<T> p; cx<float> dp; float mag; };
template <typename T, class Coef>
__device__ __forceinline__ Eval3<T> split_eval3(unsigned mask, int n, cx<T> x, float axf, Coef c) {
    const int lane = threadIdx.x % SL, B = (n + SL) / SL, k0 = lane * B;
    const int k1 = k0 + B - 1 < n ? k0 + B - 1 : n;
    const cx<float> xf = cxm<float>((float)x.x, (float)x.y);
    cx<T> q = cxm<T>(0, 0);
    cx<float> dq = cxm<float>(0.f, 0.f);
    float m = 0.f;
    for (int k = k1; k >= k0; --k) {
        const T ck = c(k);
        q = q * x + cxm<T>(ck, 0);
        if (k < n) dq = dq * xf + cxm<float>((float)(k + 1) * (float)c(k + 1), 0.f);
        m = m * axf + fabsf((float)ck);
    }
    cx<T> xp = pow_sq(x, B, [](cx<T> u, cx<T> v) { return u * v; });
    cx<float> xpf = pow_sq(xf, B, [](cx<float> u, cx<float> v) { return u * v; });
    float rp = pow_sq(axf, B, [](float u, float v) { return u * v; });
    for (int sft = 1; sft < SL; sft <<= 1) {
        cx<T> o;
        cx<float> od;
        o.x = __shfl_down_sync(mask, q.x, sft, SL);
        o.y = __shfl_down_sync(mask, q.y, sft, SL);
        od.x = __shfl_down_sync(mask, dq.x, sft, SL);
        od.y = __shfl_down_sync(mask, dq.y, sft, SL);
        const float om = __shfl_down_sync(mask, m, sft, SL);
        if ((lane & (2 * sft - 1)) == 0) { q = q + xp * o; dq = dq + xpf * od; m += rp * om; }
        xp = xp * xp;
        xpf = xpf * xpf;
        rp *= rp;
    }
    return {q, dq, m};
}

// p(z)/p'(z) by one thread alone (plain Horner), for the rare fallback of
// the polish step; the reversed polynomial at 1/z for |z| > 1.
__device__ cx<double> newton_ratio_serial(const double* a, int d, cx<double> z) {
    const bool rev = cabsv(z) > 1.0;
    const cx<double> x = rev ? cdivv(cxm<double>(1.0, 0.0), z) : z;
    cx<double> p = cxm<double>(rev ? a[0] : a[d], 0.0), dp = cxm<double>(0.0, 0.0);
    for (int k = d - 1; k >= 0; --k) {
        dp = dp * x + p;
        p = p * x + cxm<double>(rev ? a[d - k] : a[k], 0.0);
    }
    return rev ? cdivv(z * p, cscale(p, (double)d) - x * dp) : cdivv(p, dp);
}

// 1 / b in FP32 complex arithmetic (scaled, so tiny or huge b stay in range);
// {0, 0} for b = 0.
__device__ __forceinline__ cx<float> crecip_f(cx<float> b) { return cdivv(cxm<float>(1.f, 0.f), b); }

// Newton ratio p(z)/p'(z) on every lane of the root; *noise = |p(z)| is below
// its evaluation error bound.  For |z| > 1 the reversed polynomial is
// evaluated at w = 1/z = conj(z) / |z|^2 (the same code path: the coefficient
// order flips).  The quotient takes an FP32 reciprocal of the denominator:
// its relative error (about 1e-7) is that of p' already, and it avoids FP64
// divisions, the slow part of this GPU.
template <typename T>
__device__ cx<T> newton_ratio(unsigned mask, const T* a, int d, cx<T> z, bool* noise) {
    const T g = T(4 * (2 * d + 2 + 2 * SL)) * eps_of<T>::v;
    const T z2 = cabs2(z);
    const bool rev = z2 > T(1);
    const T r2 = rev ? T(1) / z2 : T(0);
    const cx<T> x = rev ? cxm<T>(z.x * r2, -z.y * r2) : z;
    const float azf = sqrtf((float)z2);
    const float axf = rev ? 1.f / azf : azf;
    const Eval3<T> e = split_eval3<T>(mask, d, x, axf, [&](int k) { return rev ? a[d - k] : a[k]; });
    cx<float> den = e.dp;
    if (rev) den = cxm<float>((float)(T(d) * e.p.x), (float)(T(d) * e.p.y)) -
                   cxm<float>((float)x.x, (float)x.y) * e.dp;
    const cx<float> inv = crecip_f(den);
    cx<T> N = (rev ? z * e.p : e.p) * cxm<T>((T)inv.x, (T)inv.y);
    const T gm = g * (T)e.mag;
    int nz = cabs2(e.p) <= gm * gm;
    N.x = __shfl_sync(mask, N.x, 0, SL);
    N.y = __shfl_sync(mask, N.y, 0, SL);
    *noise = __shfl_sync(mask, nz, 0, SL) != 0;
    return N;
}

// Aberth iterations on the shared approximations z[0..d); returns true when
// every root stopped moving.  Thread t works on root t / SL.
template <typename T>
__device__ bool aberth(const T* a, int d, cx<T>* z, int max_iter) {
    const int i = threadIdx.x / SL, lane = threadIdx.x % SL;
    bool done = i >= d;
    for (int it = 0; it < max_iter; ++it) {
        cx<T> zi = i < d ? z[i] : cxm<T>(0, 0);
        cx<T> corr = cxm<T>(0, 0);
        const unsigned am = __ballot_sync(0xffffffffu, !done);
        if (!done) {
            bool noise;
            cx<T> N = newton_ratio<T>(am, a, d, zi, &noise);
            // The Aberth sum sum_j 1/(z_i - z_j) only steers the step (near
            // convergence N S << 1 damps its error), so it is accumulated in
            // FP32 from differences taken in T; the Newton ratio N keeps T.
            // Lane l of the root adds the terms j = l (mod SL).
            float sx = 0.f, sy = 0.f;
            for (int j = lane; j < d; j += SL) {
                if (j == i) continue;
                const float dx = (float)(zi.x - z[j].x), dy = (float)(zi.y - z[j].y);
                const float m = dx * dx + dy * dy;
                if (m > 0.f) {
                    const float r = 1.f / m;
                    sx += dx * r;
                    sy -= dy * r;
                }
            }
            for (int o = 1; o < SL; o <<= 1) {
                sx += __shfl_xor_sync(am, sx, o, SL);
                sy += __shfl_xor_sync(am, sy, o, SL);
            }
            const cx<T> S = cxm<T>((T)sx, (T)sy);
            const cx<T> den = cxm<T>(1, 0) - N * S;
            // N / den with an FP32 reciprocal (den is near 1 at convergence; its
            // 1e-7 relative error only scales the step)
            const cx<float> inv = crecip_f(cxm<float>((float)den.x, (float)den.y));
            corr = N * cxm<T>((T)inv.x, (T)inv.y);
            const T huge = sizeof(T) == 8 ? T(1e60) : T(1e36);
            if (!(cabs2(corr) < huge) || (inv.x == 0.f && inv.y == 0.f)) corr = N;   // degenerate: Newton step
            const T tol = T(4) * eps_of<T>::v;
            if (noise || cabs2(corr) <= tol * tol * cabs2(zi)) done = true;
        }
        __syncthreads();
        if (i < d && lane == 0) z[i] = zi - corr;
        if (!__syncthreads_or(!done)) return true;
    }
    return false;
}

// Kernel 1: Aberth iterations, one CTA of DMAX * SL threads per polynomial.
// Writes the FP64 approximations to roots[.., 0] / roots[.., 2] and the
// convergence status.
__global__ void __launch_bounds__(DMAX * SL)
k_aberth(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
         int root_mode, double* __restrict__ roots, int32_t* __restrict__ status) {
    __shared__ double a[DMAX + 1];
    __shared__ float af[DMAX + 1];
    __shared__ cx<double> z[DMAX];
    __shared__ cx<float> zf[DMAX];
    __shared__ int hull[DMAX + 2];
    __shared__ int nhull, kmin;

    const int prob = blockIdx.x, i = threadIdx.x / SL, lane = threadIdx.x % SL;
    const int d = degrees[prob];
    const int64_t* c = coeffs + (size_t)prob * LDC;
    const int pre = status[prob];
    if (pre < 0) return;                       // rejected by the input checks
    if (d < 1 || d > DMAX) {
        if (threadIdx.x == 0) status[prob] = RFR_E_RANGE;
        return;
    }
    for (int k = threadIdx.x; k <= d; k += blockDim.x) { a[k] = (double)c[k]; af[k] = (float)c[k]; }
    __syncthreads();

    // Newton polygon: upper hull of (k, log2|a_k|) over a_k != 0.  The starting
    // points only steer the iteration, so the logs are taken once, in FP32.
    __shared__ float la[DMAX + 1];
    for (int k = threadIdx.x; k <= d; k += blockDim.x) la[k] = af[k] != 0.f ? log2f(fabsf(af[k])) : 0.f;
    __syncthreads();
    if (threadIdx.x == 0) {
        int km = 0;
        while (km < d && af[km] == 0.f) ++km;          // (float)a_k is 0 exactly when a_k is
        kmin = km;
        int h = 0;
        for (int k = km; k <= d; ++k) {
            if (af[k] == 0.f) continue;
            const float yk = la[k];
            while (h >= 2) {
                const int o = hull[h - 2], q = hull[h - 1];
                const float cr = (float)(q - o) * (yk - la[o]) - (la[q] - la[o]) * (float)(k - o);
                if (cr >= 0.f) --h; else break;
            }
            hull[h++] = k;
        }
        nhull = h;
    }
    __syncthreads();
    if (i < d && lane == 0) {
        cx<double> z0 = cxm<double>(0.0, 0.0);
        if (i >= kmin) {
            int e = 0;
            while (e + 1 < nhull - 1 && hull[e + 1] <= i) ++e;
            const int k0 = hull[e], k1 = hull[e + 1], m = k1 - k0, j = i - k0;
            const float u = exp2f((la[k0] - la[k1]) / (float)m);
            float sn, cs;
            sincospif(2.f * ((float)j + 0.25f) / (float)m + 0.22f * (float)e + 0.13f, &sn, &cs);
            z0 = cxm<double>((double)(u * cs), (double)(u * sn));
        }
        z[i] = z0;
        zf[i] = cxm<float>((float)z0.x, (float)z0.y);
    }
    __syncthreads();

    if (root_mode == RFR_ROOTS_FP32_BULK) {
        // the FP32 bulk; k_aberth64 finishes in FP64 with the polynomial spread
        // over a cluster of CTAs, and sets the status
        aberth<float>(af, d, zf, 400);
        if (i < d && lane == 0) {
            double* out = roots + ((size_t)prob * DMAX + i) * 4;
            out[0] = (double)zf[i].x; out[1] = 0.0; out[2] = (double)zf[i].y; out[3] = 0.0;
        }
        return;
    }
    const bool conv = aberth<double>(a, d, z, 600);
    if (i < d && lane == 0) {
        double* out = roots + ((size_t)prob * DMAX + i) * 4;
        out[0] = z[i].x; out[1] = 0.0; out[2] = z[i].y; out[3] = 0.0;
    }
    if (threadIdx.x == 0) {
        const bool suspect = pre == RFR_SF_SUSPECT;
        status[prob] = conv ? (suspect ? RFR_SF_SUSPECT : RFR_OK)
                            : (suspect ? RFR_E_NOT_SQUAREFREE : RFR_E_NO_CONVERGENCE);
    }
}

// Kernel 1b (FP32-bulk mode): the FP64 Aberth iterations from k_aberth's FP32
// roots, one polynomial per cluster of AC CTAs.  The FP64 evaluations are
// bound by the FP64 pipe of the SM they run on (B300's FP64 rate is small),
// so the polynomial's roots are dealt out over AC SMs: CTA r of the cluster
// owns the roots i = r (mod AC).  Every CTA keeps all approximations in its
// shared memory, double-buffered by iteration parity: an owner writes its new
// z_i (FP64, and an FP32 copy for the Aberth sum) into buffer it+1 of every
// CTA of the cluster through distributed shared memory, with its CTA's
// "still moving" flag, and one cluster barrier per iteration makes them
// visible.  The barrier also orders buffer reuse: buffer it & 1 is written
// again in iteration it + 2, after every CTA has passed the barrier of
// iteration it + 1, i.e. finished reading it.  All CTAs of a cluster read the
// same flags, so they stop at the same iteration; nothing returns early
// inside the loop.
constexpr int AC = 4;                         // CTAs per polynomial
constexpr int AR = DMAX / AC;                 // roots owned per CTA

__global__ void __cluster_dims__(AC, 1, 1) __launch_bounds__(AR * SL)
k_aberth64(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
           double* __restrict__ roots, int32_t* __restrict__ status, int max_iter) {
    namespace cg = cooperative_groups;
    __shared__ double a[DMAX + 1];
    __shared__ cx<double> zb[2][DMAX];
    __shared__ cx<float> zfb[2][DMAX];
    __shared__ int flag[2][AC];
    cg::cluster_group cl = cg::this_cluster();
    const int rank = (int)cl.block_rank();
    const int prob = blockIdx.x / AC;
    const int t = threadIdx.x / SL, lane = threadIdx.x % SL;
    const int i = rank + AC * t;                              // the root this lane works on
    const int d = degrees[prob];
    const int pre = status[prob];
    // uniform over the cluster: every CTA of it leaves here, or none does
    if (pre < 0 || d < 1 || d > DMAX) return;
    const int64_t* c = coeffs + (size_t)prob * LDC;
    double* R = roots + (size_t)prob * DMAX * 4;
    for (int k = threadIdx.x; k <= d; k += blockDim.x) a[k] = (double)c[k];
    for (int k = threadIdx.x; k < d; k += blockDim.x) {
        zb[0][k] = cxm<double>(R[4 * k], R[4 * k + 2]);
        zfb[0][k] = cxm<float>((float)R[4 * k], (float)R[4 * k + 2]);
    }
    cx<double>* zr[AC];
    cx<float>* zfr[AC];
#pragma unroll
    for (int q = 0; q < AC; ++q) {
        zr[q] = cl.map_shared_rank(&zb[0][0], q);
        zfr[q] = cl.map_shared_rank(&zfb[0][0], q);
    }
    int* fr = threadIdx.x < AC ? cl.map_shared_rank(&flag[0][0], (int)threadIdx.x) : nullptr;
    // every CTA of the cluster has started (its shared memory may be written)
    // and has loaded its copy before the first remote store
    cl.sync();
    bool done = i >= d;
    bool conv = false;
    int cur = 0;
    for (int it = 0; it < max_iter; ++it) {
        const int nxt = cur ^ 1;
        const cx<double>* z = zb[cur];
        const cx<float>* zf = zfb[cur];
        const cx<double> zi = i < d ? z[i] : cxm<double>(0.0, 0.0);
        cx<double> corr = cxm<double>(0.0, 0.0);
        const unsigned am = __ballot_sync(0xffffffffu, !done);
        if (!done) {
            bool noise;
            const cx<double> N = newton_ratio<double>(am, a, d, zi, &noise);
            // the Aberth sum in FP32 (it only steers the step, as in aberth()):
            // differences of the FP32 copies, except for roots so close that
            // those lose their digits, which take the FP64 difference
            const cx<float> zif = zf[i];
            const float azi = fabsf(zif.x) + fabsf(zif.y);
            float sx = 0.f, sy = 0.f;
            for (int j = lane; j < d; j += SL) {
                if (j == i) continue;
                float dx = zif.x - zf[j].x, dy = zif.y - zf[j].y;
                if (fabsf(dx) + fabsf(dy) < 0x1p-12f * (azi + fabsf(zf[j].x) + fabsf(zf[j].y))) {
                    dx = (float)(zi.x - z[j].x);
                    dy = (float)(zi.y - z[j].y);
                }
                const float m = dx * dx + dy * dy;
                if (m > 0.f) {
                    const float r = 1.f / m;
                    sx += dx * r;
                    sy -= dy * r;
                }
            }
            for (int o = 1; o < SL; o <<= 1) {
                sx += __shfl_xor_sync(am, sx, o, SL);
                sy += __shfl_xor_sync(am, sy, o, SL);
            }
            const cx<double> S = cxm<double>((double)sx, (double)sy);
            const cx<double> den = cxm<double>(1.0, 0.0) - N * S;
            const cx<float> inv = crecip_f(cxm<float>((float)den.x, (float)den.y));
            corr = N * cxm<double>((double)inv.x, (double)inv.y);
            if (!(cabs2(corr) < 1e60) || (inv.x == 0.f && inv.y == 0.f)) corr = N;   // degenerate: Newton step
            const double tol = 4.0 * eps_of<double>::v;
            if (noise || cabs2(corr) <= tol * tol * cabs2(zi)) done = true;
        }
        // every owned root (moving or not) goes into buffer nxt of every CTA
        if (i < d && lane == 0) {
            const cx<double> zn = zi - corr;
            const cx<float> znf = cxm<float>((float)zn.x, (float)zn.y);
#pragma unroll
            for (int q = 0; q < AC; ++q) {
                zr[q][nxt * DMAX + i] = zn;
                zfr[q][nxt * DMAX + i] = znf;
            }
        }
        const int moving = __syncthreads_or(!done);
        if (threadIdx.x < AC) fr[nxt * AC + rank] = moving;
        cl.sync();
        int any = 0;
#pragma unroll
        for (int q = 0; q < AC; ++q) any |= flag[nxt][q];
        cur = nxt;
        if (!any) { conv = true; break; }
    }
    if (i < d && lane == 0) {
        double* out = R + (size_t)i * 4;
        out[0] = zb[cur][i].x; out[1] = 0.0; out[2] = zb[cur][i].y; out[3] = 0.0;
    }
    if (rank == 0 && threadIdx.x == 0) {
        const bool suspect = pre == RFR_SF_SUSPECT;
        status[prob] = conv ? (suspect ? RFR_SF_SUSPECT : RFR_OK)
                            : (suspect ? RFR_E_NOT_SQUAREFREE : RFR_E_NO_CONVERGENCE);
    }
}

// Steps 3 and 4 take SL = 8 lanes per root, RPC roots of one polynomial per
// CTA: blockIdx.x = problem * (DMAX / RPC) + chunk.  Both are bound by the
// FP64 pipe of the SMs they run on, so a small batch takes 4 roots per CTA
// (one warp; a degree-100 polynomial spread over 25 SMs) and a large one 16.
// A polynomial is evaluated by a split Horner scheme: lane l of a root sums
// the B = ceil((d+1)/SL) coefficients k in [lB, lB + B) as
// q_l(z) = sum a_k z^(k - lB) (Horner), and a shuffle tree forms
// p(z) = sum_l z^(lB) q_l(z) with the powers z^(sB), s = 1, 2, 4.  The chain
// is about d / SL steps plus the power's log2 B squarings, and the total work
// stays about d steps per root.
struct RootWarp { int prob, d, i, lane; };
template <int RPC>
__device__ __forceinline__ bool root_warp(const int32_t* degrees, const int32_t* status, RootWarp* r) {
    constexpr int RCHUNKS = DMAX / RPC;
    r->prob = blockIdx.x / RCHUNKS;
    r->d = degrees[r->prob];
    r->lane = threadIdx.x % SL;
    r->i = (blockIdx.x % RCHUNKS) * RPC + (int)threadIdx.x / SL;
    const int st = status[r->prob];
    return (st == RFR_OK || st == RFR_SF_SUSPECT) && r->d >= 1 && r->d <= DMAX &&
           (blockIdx.x % RCHUNKS) * RPC < r->d;
}

__device__ __forceinline__ cdd shfl_down_cdd(cdd v, int s) {
    v.re.hi = __shfl_down_sync(0xffffffffu, v.re.hi, s, SL);
    v.re.lo = __shfl_down_sync(0xffffffffu, v.re.lo, s, SL);
    v.im.hi = __shfl_down_sync(0xffffffffu, v.im.hi, s, SL);
    v.im.lo = __shfl_down_sync(0xffffffffu, v.im.lo, s, SL);
    return v;
}

// sum_{k=0}^{n} c(k) Z^k in double-double, split over the root's SL lanes; its
// lane 0 returns it.
template <class Coef>
__device__ cdd warp_poly_dd(int n, cdd Z, Coef c) {
    const int lane = threadIdx.x % SL, B = (n + SL) / SL, k0 = lane * B;
    const int k1 = k0 + B - 1 < n ? k0 + B - 1 : n;
    cdd q = cdd_make(0.0, 0.0);
    if (k0 <= n) {
        q = cdd_make(c(k1), 0.0);
        for (int k = k1 - 1; k >= k0; --k) q = cdd_add_d(cdd_mul(q, Z), c(k));
    }
    cdd zp = pow_sq(Z, B, [](cdd u, cdd v) { return cdd_mul(u, v); });
    for (int s = 1; s < SL; s <<= 1) {
        const cdd o = shfl_down_cdd(q, s);
        if ((lane & (2 * s - 1)) == 0) q = cdd_add(q, cdd_mul(zp, o));
        zp = cdd_mul(zp, zp);
    }
    return q;
}

// The same in FP64 complex arithmetic.
template <class Coef>
__device__ cx<double> warp_poly_c(int n, cx<double> z, Coef c) {
    const int lane = threadIdx.x % SL, B = (n + SL) / SL, k0 = lane * B;
    const int k1 = k0 + B - 1 < n ? k0 + B - 1 : n;
    cx<double> q = cxm<double>(0.0, 0.0);
    if (k0 <= n) {
        q = cxm<double>(c(k1), 0.0);
        for (int k = k1 - 1; k >= k0; --k) q = q * z + cxm<double>(c(k), 0.0);
    }
    cx<double> zp = pow_sq(z, B, [](cx<double> u, cx<double> v) { return u * v; });
    for (int s = 1; s < SL; s <<= 1) {
        cx<double> o;
        o.x = __shfl_down_sync(0xffffffffu, q.x, s, SL);
        o.y = __shfl_down_sync(0xffffffffu, q.y, s, SL);
        if ((lane & (2 * s - 1)) == 0) q = q + zp * o;
        zp = zp * zp;
    }
    return q;
}

// sum_{k=0}^{n} c(k) r^k for real r >= 0, split the same way.
template <class Coef>
__device__ double warp_poly_r(int n, double r, Coef c) {
    const int lane = threadIdx.x % SL, B = (n + SL) / SL, k0 = lane * B;
    const int k1 = k0 + B - 1 < n ? k0 + B - 1 : n;
    double q = 0.0;
    if (k0 <= n) {
        q = c(k1);
        for (int k = k1 - 1; k >= k0; --k) q = q * r + c(k);
    }
    double rp = pow_sq(r, B, [](double u, double v) { return u * v; });
    for (int s = 1; s < SL; s <<= 1) {
        const double o = __shfl_down_sync(0xffffffffu, q, s, SL);
        if ((lane & (2 * s - 1)) == 0) q += rp * o;
        rp *= rp;
    }
    return q;
}

// Kernel 2: Newton steps with p evaluated in double-double (the correction
// itself in FP64), so each root becomes a DD value: one step, or up to five
// for a root close to another (below).
template <int RPC>
__global__ void __launch_bounds__(RPC * SL)
k_polish(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
         const int32_t* __restrict__ status, double* __restrict__ roots) {
    __shared__ double a[DMAX + 1];
    __shared__ cx<float> zs[DMAX];                           // FP32 copies of the roots
    RootWarp R;
    if (!root_warp<RPC>(degrees, status, &R)) return;         // uniform over the CTA
    const int d = R.d, i = R.i;
    const int64_t* c = coeffs + (size_t)R.prob * LDC;
    const double* Rt = roots + (size_t)R.prob * DMAX * 4;
    for (int k = threadIdx.x; k <= d; k += blockDim.x) a[k] = (double)c[k];
    for (int k = threadIdx.x; k < d; k += blockDim.x) zs[k] = cxm<float>((float)Rt[4 * k], (float)Rt[4 * k + 2]);
    __syncthreads();
    // lanes of roots past the degree compute on the last root and write nothing
    // (every lane of the warp takes part in the shuffles)
    const bool live = i < d;
    const int ii = live ? i : d - 1;
    double* out = roots + ((size_t)R.prob * DMAX + ii) * 4;
    cdd Z = {{out[0], out[1]}, {out[2], out[3]}};
    // squared distance to the nearest other root (FP32, lanes over j)
    float dmin2 = INFINITY;
    for (int j = R.lane; j < d; j += SL) {
        if (j == ii) continue;
        const float dx = zs[ii].x - zs[j].x, dy = zs[ii].y - zs[j].y;
        dmin2 = fminf(dmin2, dx * dx + dy * dy);
    }
    for (int o = SL / 2; o; o >>= 1) dmin2 = fminf(dmin2, __shfl_xor_sync(0xffffffffu, dmin2, o, SL));
    // Newton steps with p in double-double (the correction itself in FP64).
    // From the FP64 Aberth root (error ~1e-16 |z|) one step squares the error,
    // and that is the common case.  A root whose step was not tiny against the
    // distance to its nearest neighbour (close roots, where the FP64 root is
    // accurate only to a fraction of that distance) takes further steps, each
    // squaring its error, up to five in all.  The inclusion radius computed
    // afterwards certifies what they reached.
    for (int step = 0; step < 5; ++step) {
        const cx<double> zh = cxm<double>(Z.re.hi, Z.im.hi);
        const bool rev = cabsv(zh) > 1.0;
        // |z| > 1: P(w) = w^d p(1/w) = sum_m a_{d-m} w^m at w = 1/z.  The evaluation
        // is the same call either way (the lanes of a warp hold different roots).
        const cdd X = rev ? cdd_inv(Z) : Z;
        const cx<double> xh = cxm<double>(X.re.hi, X.im.hi);
        const cdd P = warp_poly_dd(d, X, [&](int k) { return a[rev ? d - k : k]; });
        const cx<double> dP = warp_poly_c(d - 1, xh, [&](int m) { return (double)(m + 1) * a[rev ? d - m - 1 : m + 1]; });
        const cx<double> Ph = cxm<double>(P.re.hi, P.im.hi);
        cx<double> N = rev ? cdivv(zh * Ph, cscale(Ph, (double)d) - xh * dP) : cdivv(Ph, dP);
        if (R.lane == 0) {
            if (!(cabsv(N) < 1e300)) N = newton_ratio_serial(a, d, zh);   // degenerate: plain FP64 Newton ratio
            Z.re = dd_add_d(Z.re, -N.x);
            Z.im = dd_add_d(Z.im, -N.y);
        }
        // the root's lanes take the new approximation and its step size from its first lane
        Z.re.hi = __shfl_sync(0xffffffffu, Z.re.hi, 0, SL);
        Z.re.lo = __shfl_sync(0xffffffffu, Z.re.lo, 0, SL);
        Z.im.hi = __shfl_sync(0xffffffffu, Z.im.hi, 0, SL);
        Z.im.lo = __shfl_sync(0xffffffffu, Z.im.lo, 0, SL);
        const double n2 = __shfl_sync(0xffffffffu, cabs2(N), 0, SL);
        const bool more = live && n2 > 1e-12 * (double)dmin2;      // |step| > 1e-6 x nearest distance
        if (!__any_sync(0xffffffffu, more)) break;
    }
    if (R.lane == 0 && live) {
        out[0] = Z.re.hi; out[1] = Z.re.lo; out[2] = Z.im.hi; out[3] = Z.im.lo;
    }
}

// Kernel 3: inclusion radius r_i = d |p(z_i)| / prod_{j != i} |z_i - z_j| with
// |p(z_i)| from a double-double evaluation plus its error bound.
template <int RPC>
__global__ void __launch_bounds__(RPC * SL)
k_radius(const int64_t* __restrict__ coeffs, const int32_t* __restrict__ degrees,
         const int32_t* __restrict__ status, const double* __restrict__ roots,
         double* __restrict__ radius) {
    __shared__ double a[DMAX + 1];
    __shared__ cx<double> z[DMAX];
    RootWarp R;
    if (!root_warp<RPC>(degrees, status, &R)) return;         // uniform over the CTA
    const int d = R.d, i = R.i;
    const int64_t* c = coeffs + (size_t)R.prob * LDC;
    const double* Rt = roots + (size_t)R.prob * DMAX * 4;
    for (int k = threadIdx.x; k <= d; k += blockDim.x) a[k] = (double)c[k];
    for (int k = threadIdx.x; k < d; k += blockDim.x) z[k] = cxm<double>(Rt[4 * k], Rt[4 * k + 2]);
    __syncthreads();
    // lanes of roots past the degree compute on the last root and write nothing
    // (every lane of the warp takes part in the shuffles)
    const bool live = i < d;
    const int ii = live ? i : d - 1;
    const cdd Z = {{Rt[4 * ii], Rt[4 * ii + 1]}, {Rt[4 * ii + 2], Rt[4 * ii + 3]}};
    const cx<double> zh = z[ii];
    const double az = cabsv(zh);
    const bool rev = az > 1.0;
    // |z| > 1: |p(z)| = |z|^d |P(1/z)| (same call either way, as in k_polish)
    const cdd X = rev ? cdd_inv(Z) : Z;
    const cdd P = warp_poly_dd(d, X, [&](int k) { return a[rev ? d - k : k]; });
    const double mag = warp_poly_r(d, rev ? 1.0 / az : az, [&](int k) { return fabs(a[rev ? d - k : k]); });
    const double pv = hypot(P.re.hi, P.im.hi);
    const double err = (double)(2 * d + 8) * 0x1p-100 * mag;
    const double lp = (rev ? (double)d * log2(az) : 0.0) + log2(pv + err);
    // log2 of prod_{j != i} |z_i - z_j| in FP32 (d <= 128 terms, each with
    // relative error ~1e-7: the sum is within 2e-5 of the exact value,
    // far inside the 1.01 safety factor below), lanes over j
    float lprodf = 0.f;
    bool coincide = false;
    for (int j = R.lane; j < d; j += SL) {
        if (j == ii) continue;
        const float dist = (float)cabsv(zh - z[j]);
        if (!(dist > 0.f)) coincide = true; else lprodf += log2f(dist);
    }
    int co = coincide ? 1 : 0;
    for (int o = SL / 2; o; o >>= 1) {
        lprodf += __shfl_xor_sync(0xffffffffu, lprodf, o, SL);
        co |= __shfl_xor_sync(0xffffffffu, co, o, SL);
    }
    coincide = co != 0;
    if (R.lane == 0 && live) {
        const double lprod = (double)lprodf;
        double r = coincide ? INFINITY : exp2(log2((double)d) + lp - lprod) * 1.01 + 0x1p-96 * az;
        if (d == 1) r = 0x1p-96 * az + 0x1p-100;
        radius[(size_t)R.prob * DMAX + i] = r;
    }
}

}  // namespace rfr

using namespace rfr;

extern "C" int rfr_stage_roots(const int64_t* coeffs, const int32_t* degrees, int batch,
                               int root_mode, double* roots, double* radius,
                               int32_t* status, void* stream) {
    if (batch < 0 || !coeffs || !degrees || !roots || !radius || !status) return RFR_E_INVALID;
    if (batch == 0) return RFR_OK;
    cudaStream_t s = (cudaStream_t)stream;
    k_aberth<<<batch, DMAX * SL, 0, s>>>(coeffs, degrees, root_mode, roots, status);
    if (root_mode == RFR_ROOTS_FP32_BULK) k_aberth64<<<batch * AC, AR * SL, 0, s>>>(coeffs, degrees, roots, status, 200);
    if (batch <= 16) {
        k_polish<4><<<batch * (DMAX / 4), 4 * SL, 0, s>>>(coeffs, degrees, status, roots);
        k_radius<4><<<batch * (DMAX / 4), 4 * SL, 0, s>>>(coeffs, degrees, status, roots, radius);
    } else {
        k_polish<16><<<batch * (DMAX / 16), 16 * SL, 0, s>>>(coeffs, degrees, status, roots);
        k_radius<16><<<batch * (DMAX / 16), 16 * SL, 0, s>>>(coeffs, degrees, status, roots, radius);
    }
    return cudaGetLastError() == cudaSuccess ? RFR_OK : RFR_E_CUDA;
}
