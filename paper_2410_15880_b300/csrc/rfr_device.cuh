// rfr_device.cuh — device-side helpers shared by the RFR kernels:
// double-double (DD) arithmetic, complex FP64/DD helpers, fixed-point
// conversion, launch-side declarations.
//
// Double-double arithmetic follows the published error-free transformations:
// Knuth's TwoSum, Dekker's FastTwoSum, and the FMA form of Dekker's TwoProduct
// (the product's rounding error is fma(a, b, -a*b) exactly), combined the way
// Hida, Li and Bailey describe for their double-double type.  A DD value
// hi + lo carries about 106 significant bits.
#pragma once
#include <cstdint>
#include <cuda_runtime.h>
#include "../../include/rfr_stages.h"

namespace rfr {

constexpr int DMAX = RFR_MAX_DEGREE;
constexpr int LDC = RFR_LDC;

struct dd { double hi, lo; };
struct cdd { dd re, im; };

__host__ __device__ __forceinline__ dd dd_make(double x) { return {x, 0.0}; }

// Knuth TwoSum: s + e == a + b exactly.
__host__ __device__ __forceinline__ dd two_sum(double a, double b) {
    double s = a + b;
    double bb = s - a;
    double e = (a - (s - bb)) + (b - bb);
    return {s, e};
}
// Dekker FastTwoSum, valid when |a| >= |b| (or a == 0).
__host__ __device__ __forceinline__ dd fast_two_sum(double a, double b) {
    double s = a + b;
    double e = b - (s - a);
    return {s, e};
}
// TwoProduct with FMA: p + e == a * b exactly.
__device__ __forceinline__ dd two_prod(double a, double b) {
    double p = a * b;
    double e = fma(a, b, -p);
    return {p, e};
}
__device__ __forceinline__ dd dd_add(dd a, dd b) {
    dd s = two_sum(a.hi, b.hi);
    dd t = two_sum(a.lo, b.lo);
    s.lo += t.hi;
    s = fast_two_sum(s.hi, s.lo);
    s.lo += t.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_neg(dd a) { return {-a.hi, -a.lo}; }
__device__ __forceinline__ dd dd_sub(dd a, dd b) { return dd_add(a, dd_neg(b)); }
__device__ __forceinline__ dd dd_add_d(dd a, double b) {
    dd s = two_sum(a.hi, b);
    s.lo += a.lo;
    return fast_two_sum(s.hi, s.lo);
}
__device__ __forceinline__ dd dd_mul(dd a, dd b) {
    dd p = two_prod(a.hi, b.hi);
    p.lo += a.hi * b.lo + a.lo * b.hi;
    return fast_two_sum(p.hi, p.lo);
}
__device__ __forceinline__ dd dd_mul_d(dd a, double b) {
    dd p = two_prod(a.hi, b);
    p.lo += a.lo * b;
    return fast_two_sum(p.hi, p.lo);
}
// a / b by long division in three FP64 steps (quotient digits q1, q2, q3).
__device__ __forceinline__ dd dd_div(dd a, dd b) {
    double q1 = a.hi / b.hi;
    dd r = dd_sub(a, dd_mul_d(b, q1));
    double q2 = r.hi / b.hi;
    r = dd_sub(r, dd_mul_d(b, q2));
    double q3 = r.hi / b.hi;
    dd q = fast_two_sum(q1, q2);
    return dd_add_d(q, q3);
}

__device__ __forceinline__ cdd cdd_make(double re, double im) { return {{re, 0.0}, {im, 0.0}}; }
__device__ __forceinline__ cdd cdd_add(cdd a, cdd b) { return {dd_add(a.re, b.re), dd_add(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_sub(cdd a, cdd b) { return {dd_sub(a.re, b.re), dd_sub(a.im, b.im)}; }
__device__ __forceinline__ cdd cdd_mul(cdd a, cdd b) {
    return {dd_sub(dd_mul(a.re, b.re), dd_mul(a.im, b.im)),
            dd_add(dd_mul(a.re, b.im), dd_mul(a.im, b.re))};
}
__device__ __forceinline__ cdd cdd_add_d(cdd a, double b) { return {dd_add_d(a.re, b), a.im}; }
// 1 / z = conj(z) / |z|^2 in DD.
__device__ __forceinline__ cdd cdd_inv(cdd z) {
    dd m = dd_add(dd_mul(z.re, z.re), dd_mul(z.im, z.im));
    return {dd_div(z.re, m), dd_neg(dd_div(z.im, m))};
}

// ---- complex FP64 -----------------------------------------------------
__device__ __forceinline__ double2 c_add(double2 a, double2 b) { return make_double2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ double2 c_sub(double2 a, double2 b) { return make_double2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ double2 c_mul(double2 a, double2 b) {
    return make_double2(fma(a.x, b.x, -a.y * b.y), fma(a.x, b.y, a.y * b.x));
}
__device__ __forceinline__ double c_abs(double2 a) { return hypot(a.x, a.y); }
__device__ __forceinline__ double2 c_div(double2 a, double2 b) {
    // scaled to avoid overflow in |b|^2
    double s = fmax(fabs(b.x), fabs(b.y));
    if (s == 0.0) return make_double2(0.0, 0.0);
    double bx = b.x / s, by = b.y / s;
    double m = bx * bx + by * by;
    return make_double2((a.x * bx + a.y * by) / (m * s), (a.y * bx - a.x * by) / (m * s));
}

// ---- fixed point --------------------------------------------------------
// round(frac(x) * 2^64) mod 2^64 for a DD value x with |x| < 2^52.
__device__ __forceinline__ uint64_t dd_frac_fixed64(dd x) {
    double fl = floor(x.hi);
    // x.hi - fl is not exact when -1 < x.hi < 0 (it is x.hi + 1): keep its
    // rounding error with TwoSum, then add x.lo.  f lies in (-tiny, 1 + tiny).
    dd t = two_sum(x.hi, -fl);
    dd f = two_sum(t.hi, t.lo + x.lo);
    double X = ldexp(f.hi, 64);                // exact scaling
    double Y = ldexp(f.lo, 64);
    double Xi = floor(X);
    double Xf = X - Xi;                        // exact, in [0, 1)
    if (Xi >= 9223372036854775808.0) Xi -= 18446744073709551616.0;   // bring into int64 range, mod 2^64
    if (Xi < -9223372036854775808.0) Xi += 18446744073709551616.0;
    long long r = llrint(Xf + Y);              // |Y| <= 2^-42 * |X|: Xf + Y is within int range
    return (uint64_t)(long long)Xi + (uint64_t)r;
}

__device__ __forceinline__ uint64_t circ_dist(uint64_t y) { return y <= (0ull - y) ? y : (0ull - y); }

}  // namespace rfr
