// general.cu — any nonzero p in Z[x] (Section 2's reductions to the monic,
// square-free case), host code around the GPU factorisation:
//   1. content and sign: p = content * pp, pp primitive with lc(pp) > 0;
//   2. the power of x that divides pp;
//   3. Yun's square-free decomposition pp = prod_i a_i^i, computed modulo
//      61-bit primes (gcds over F_l; primes whose gcd(pp, pp') has more
//      than the smallest degree seen are discarded), lifted by the Chinese
//      remainder theorem to the symmetric range and checked exactly:
//      prod_i a_i^i == pp in 128-bit integers;
//   4. (rfr_factor_general) the monic transform of every part:
//      q_i(y) = lc_i^(e-1) a_i(y / lc_i) is monic and square-free in Z[y];
//      all of them are factored as one batch by the GPU path;
//   5. every monic factor g(y) of q_i maps back to the primitive part of
//      g(lc_i x), a factor of pp with multiplicity i, and
//      content * prod f^m == p is checked exactly.
#include <algorithm>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <vector>
#include "rfr.h"

namespace {

typedef __int128 i128;
typedef unsigned __int128 u128;
typedef std::vector<uint64_t> PolyM;     // coefficients modulo a prime, ascending, trimmed
typedef std::vector<i128> PolyZ;         // integer coefficients, ascending, trimmed

const uint64_t PRIMES[] = {             // the six largest primes below 2^61 (the first is 2^61 - 1)
    2305843009213693951ull, 2305843009213693921ull, 2305843009213693907ull,
    2305843009213693723ull, 2305843009213693693ull, 2305843009213693669ull,
};
const int NPRIMES = sizeof(PRIMES) / sizeof(PRIMES[0]);

struct Mod {
    uint64_t l;
    uint64_t add(uint64_t a, uint64_t b) const { uint64_t s = a + b; return s >= l ? s - l : s; }
    uint64_t sub(uint64_t a, uint64_t b) const { return a >= b ? a - b : a + l - b; }
    uint64_t mul(uint64_t a, uint64_t b) const { return (uint64_t)((u128)a * b % l); }
    uint64_t pow(uint64_t a, uint64_t e) const {
        uint64_t r = 1;
        for (; e; e >>= 1, a = mul(a, a)) if (e & 1) r = mul(r, a);
        return r;
    }
    uint64_t inv(uint64_t a) const { return pow(a, l - 2); }
    uint64_t from(i128 v) const { i128 r = v % (i128)l; return (uint64_t)(r < 0 ? r + (i128)l : r); }
};

void trim(PolyM& a) { while (!a.empty() && a.back() == 0) a.pop_back(); }
void trimz(PolyZ& a) { while (!a.empty() && a.back() == 0) a.pop_back(); }
int deg(const PolyM& a) { return (int)a.size() - 1; }

PolyM deriv(const Mod& M, const PolyM& a) {
    PolyM d;
    for (size_t k = 1; k < a.size(); ++k) d.push_back(M.mul(a[k], k % M.l));
    trim(d);
    return d;
}

PolyM psub(const Mod& M, const PolyM& a, const PolyM& b) {
    PolyM r(std::max(a.size(), b.size()), 0);
    for (size_t k = 0; k < r.size(); ++k)
        r[k] = M.sub(k < a.size() ? a[k] : 0, k < b.size() ? b[k] : 0);
    trim(r);
    return r;
}

// a = q b + r with deg r < deg b (b nonzero)
void divmod(const Mod& M, PolyM a, const PolyM& b, PolyM* q, PolyM* r) {
    const int db = deg(b);
    const uint64_t il = M.inv(b.back());
    PolyM qq(a.size() > b.size() ? a.size() - b.size() + 1 : 1, 0);
    for (int k = deg(a); k >= db; --k) {
        const uint64_t c = M.mul(a[k], il);
        qq[k - db] = c;
        if (c)
            for (int j = 0; j <= db; ++j) a[k - db + j] = M.sub(a[k - db + j], M.mul(c, b[j]));
    }
    trim(a);
    trim(qq);
    if (q) *q = qq;
    if (r) *r = a;
}

PolyM monic(const Mod& M, PolyM a) {
    if (a.empty()) return a;
    const uint64_t il = M.inv(a.back());
    for (auto& c : a) c = M.mul(c, il);
    return a;
}

PolyM gcd(const Mod& M, PolyM a, PolyM b) {
    while (!b.empty()) {
        PolyM r;
        divmod(M, a, b, nullptr, &r);
        a.swap(b);
        b.swap(r);
    }
    return monic(M, a);
}

PolyM exact_div(const Mod& M, const PolyM& a, const PolyM& b) {
    PolyM q;
    divmod(M, a, b, &q, nullptr);
    return q;
}

// Yun's algorithm over F_l for a monic f with l > deg f: parts[i-1] = a_i.
std::vector<PolyM> yun(const Mod& M, const PolyM& f) {
    std::vector<PolyM> parts;
    const PolyM fp = deriv(M, f);
    const PolyM g = gcd(M, f, fp);
    PolyM b = exact_div(M, f, g);
    PolyM c = exact_div(M, fp, g);
    PolyM d = psub(M, c, deriv(M, b));
    for (int guard = 0; deg(b) >= 1 && guard <= RFR_MAX_DEGREE; ++guard) {
        const PolyM a = gcd(M, b, d);
        parts.push_back(a);
        b = exact_div(M, b, a);
        c = exact_div(M, d, a);
        d = psub(M, c, deriv(M, b));
    }
    return parts;
}

i128 abs128(i128 v) { return v < 0 ? -v : v; }

bool mul_ovf(const PolyZ& a, const PolyZ& b, PolyZ* out) {
    PolyZ r(a.size() + b.size() - 1, 0);
    for (size_t i = 0; i < a.size(); ++i)
        for (size_t j = 0; j < b.size(); ++j) {
            i128 t;
            if (__builtin_mul_overflow(a[i], b[j], &t)) return false;
            if (__builtin_add_overflow(r[i + j], t, &r[i + j])) return false;
        }
    *out = r;
    return true;
}

i128 gcd128(i128 a, i128 b) {
    a = abs128(a); b = abs128(b);
    while (b) { i128 t = a % b; a = b; b = t; }
    return a;
}

// Primitive part with a positive leading coefficient.
void primitive(PolyZ& a) {
    i128 g = 0;
    for (auto c : a) g = gcd128(g, c);
    if (g == 0) return;
    if (a.back() < 0) g = -g;
    for (auto& c : a) c /= g;
}

struct Part { PolyZ f; int mult; };

// Steps 1, 2 and 4: content, x^k, Yun.  The parts are the primitive a_i of
// pp (lc > 0).  Yun runs modulo primes on pp made monic (primes dividing
// lc(pp) are skipped); lc(pp) * a_i / lc(a_i) is an integer polynomial, so
// lc(pp) times the monic part modulo the primes lifts to it, and its
// primitive part is a_i.
int decompose(const int64_t* coeffs, int degree, int64_t* content, int* xpow, std::vector<Part>* parts) {
    if (!coeffs || degree < 0 || degree > RFR_MAX_DEGREE) return RFR_E_INVALID;
    int D = degree;
    while (D >= 0 && coeffs[D] == 0) --D;
    if (D < 0) return RFR_E_INVALID;                      // the zero polynomial
    i128 g = 0;
    for (int k = 0; k <= D; ++k) g = gcd128(g, coeffs[k]);
    if (coeffs[D] < 0) g = -g;
    *content = (int64_t)g;
    int lo = 0;
    while (coeffs[lo] == 0) ++lo;
    *xpow = lo;
    PolyZ pp;
    for (int k = lo; k <= D; ++k) pp.push_back((i128)coeffs[k] / g);
    const int Dp = (int)pp.size() - 1;
    const i128 lc = pp.back();
    parts->clear();
    if (Dp == 0) return RFR_OK;
    // Yun modulo several primes; keep the decompositions whose gcd(pp, pp')
    // has the smallest degree, lift the first two that agree.
    std::vector<std::vector<PolyM>> dec(NPRIMES);
    std::vector<int> gdeg(NPRIMES, 1 << 30);
    for (int t = 0; t < NPRIMES; ++t) {
        const Mod M{PRIMES[t]};
        if (M.from(lc) == 0) continue;
        PolyM f(Dp + 1);
        for (int k = 0; k <= Dp; ++k) f[k] = M.from(pp[k]);
        dec[t] = yun(M, monic(M, f));
        int s = 0;
        for (size_t i = 0; i < dec[t].size(); ++i) s += (int)i * deg(dec[t][i]);
        gdeg[t] = s;
    }
    const int best = *std::min_element(gdeg.begin(), gdeg.end());
    auto pattern = [&](int t) {
        std::vector<int> d;
        for (auto& a : dec[t]) d.push_back(deg(a));
        return d;
    };
    int t1 = -1, t2 = -1;
    for (int t = 0; t < NPRIMES && t2 < 0; ++t) {
        if (gdeg[t] != best) continue;
        if (t1 < 0) t1 = t;
        else if (pattern(t) == pattern(t1)) t2 = t;
    }
    if (t2 < 0) return RFR_E_OVERFLOW;
    const Mod M1{PRIMES[t1]}, M2{PRIMES[t2]};
    const u128 Mprod = (u128)M1.l * M2.l;
    const uint64_t inv1 = M2.inv(M1.l % M2.l);
    const uint64_t lc1 = M1.from(lc), lc2 = M2.from(lc);
    PolyZ prod(1, 1);
    for (size_t i = 0; i < dec[t1].size(); ++i) {
        const PolyM& a1 = dec[t1][i];
        const PolyM& a2 = dec[t2][i];
        PolyZ a(a1.size());
        for (size_t k = 0; k < a1.size(); ++k) {
            const uint64_t r1 = M1.mul(a1[k], lc1), r2 = M2.mul(a2[k], lc2);
            const uint64_t h = M2.mul(M2.sub(r2, r1 % M2.l), inv1);
            const u128 x = (u128)r1 + (u128)M1.l * h;
            a[k] = x > Mprod / 2 ? (i128)x - (i128)Mprod : (i128)x;
        }
        primitive(a);
        for (int m = 0; m <= (int)i; ++m)
            if (!mul_ovf(prod, a, &prod)) return RFR_E_OVERFLOW;
        if (a.size() > 1) parts->push_back({a, (int)i + 1});
    }
    trimz(prod);
    if (prod != pp) return RFR_E_OVERFLOW;                // a lift left the symmetric range
    return RFR_OK;
}

// Step 3 for one part: q(y) = lc^(e-1) a(y / lc), monic; false if a
// coefficient reaches 2^53 (the GPU path's input range).
bool monic_transform(const PolyZ& a, std::vector<int64_t>* q) {
    const int e = (int)a.size() - 1;
    const i128 lc = a.back();
    q->assign(e + 1, 0);
    (*q)[e] = 1;
    for (int k = 0; k < e; ++k) {
        i128 v = a[k];
        for (int t = 0; t < e - 1 - k; ++t)
            if (__builtin_mul_overflow(v, lc, &v)) return false;
        if (abs128(v) >= ((i128)1 << 53)) return false;
        (*q)[k] = (int64_t)v;
    }
    return true;
}

// g(y) monic factor of q -> primitive part of g(lc x); false on overflow
bool back_transform(const PolyZ& g, i128 lc, PolyZ* out) {
    PolyZ h(g.size());
    i128 p = 1;
    for (size_t k = 0; k < g.size(); ++k) {
        if (__builtin_mul_overflow(g[k], p, &h[k])) return false;
        if (k + 1 < g.size() && __builtin_mul_overflow(p, lc, &p)) return false;
    }
    primitive(h);
    for (auto c : h) if (abs128(c) >= ((i128)1 << 63)) return false;
    *out = h;
    return true;
}

bool less_factor(const Part& a, const Part& b) {
    if (a.f.size() != b.f.size()) return a.f.size() < b.f.size();
    for (size_t k = 0; k + 1 < a.f.size(); ++k)
        if (a.f[k] != b.f[k]) return a.f[k] < b.f[k];
    if (a.f.back() != b.f.back()) return a.f.back() < b.f.back();
    return a.mult < b.mult;
}

int fill(std::vector<Part>& fs, int64_t content, rfr_factorization* out) {
    std::sort(fs.begin(), fs.end(), less_factor);
    size_t total = 0;
    for (auto& f : fs) total += f.f.size();
    out->content = content;
    out->n_factors = (int)fs.size();
    out->degrees = (int*)malloc(sizeof(int) * (fs.size() + 1));
    out->multiplicities = (int*)malloc(sizeof(int) * (fs.size() + 1));
    out->coeffs = (int64_t*)malloc(sizeof(int64_t) * (total + 1));
    if (!out->degrees || !out->multiplicities || !out->coeffs) {
        rfr_factorization_free(out);
        return RFR_E_OOM;
    }
    size_t o = 0;
    for (size_t i = 0; i < fs.size(); ++i) {
        out->degrees[i] = (int)fs[i].f.size() - 1;
        out->multiplicities[i] = fs[i].mult;
        for (auto c : fs[i].f) out->coeffs[o++] = (int64_t)c;
    }
    return RFR_OK;
}

// content * prod f^m == p, exactly
bool product_check(const std::vector<Part>& fs, int64_t content, const int64_t* coeffs, int degree) {
    PolyZ prod(1, (i128)content);
    for (auto& f : fs)
        for (int m = 0; m < f.mult; ++m)
            if (!mul_ovf(prod, f.f, &prod)) return false;
    PolyZ p(coeffs, coeffs + degree + 1);
    trimz(p);
    trimz(prod);
    return prod == p;
}

}  // namespace

extern "C" void rfr_factorization_free(rfr_factorization* f) {
    if (!f) return;
    free(f->degrees);
    free(f->multiplicities);
    free(f->coeffs);
    memset(f, 0, sizeof(*f));
}

extern "C" int rfr_squarefree(const int64_t* coeffs, int degree, rfr_factorization* out) {
    if (!out) return RFR_E_INVALID;
    memset(out, 0, sizeof(*out));
    int64_t content;
    int xpow;
    std::vector<Part> parts;
    int st = decompose(coeffs, degree, &content, &xpow, &parts);
    if (st != RFR_OK) return st;
    std::vector<Part> fs;
    if (xpow) fs.push_back({PolyZ{0, 1}, xpow});
    for (auto& a : parts) {
        for (auto c : a.f) if (abs128(c) >= ((i128)1 << 63)) return RFR_E_OVERFLOW;
        fs.push_back(a);
    }
    if (!product_check(fs, content, coeffs, degree)) return RFR_E_OVERFLOW;
    return fill(fs, content, out);
}

extern "C" int rfr_factor_general(rfr_ctx* ctx, const int64_t* coeffs, int degree, rfr_factorization* out) {
    if (!ctx || !out) return RFR_E_INVALID;
    memset(out, 0, sizeof(*out));
    int64_t content;
    int xpow;
    std::vector<Part> parts;
    int st = decompose(coeffs, degree, &content, &xpow, &parts);
    if (st != RFR_OK) return st;
    // every square-free part, made monic, in one GPU batch
    std::vector<std::vector<int64_t>> in(parts.size());
    std::vector<const int64_t*> ptrs(parts.size());
    std::vector<int> degs(parts.size());
    for (size_t i = 0; i < parts.size(); ++i) {
        if (!monic_transform(parts[i].f, &in[i])) return RFR_E_RANGE;
        ptrs[i] = in[i].data();
        degs[i] = (int)in[i].size() - 1;
    }
    std::vector<Part> fs;
    if (xpow) fs.push_back({PolyZ{0, 1}, xpow});
    if (!parts.empty()) {
        std::vector<rfr_factors> res(parts.size());
        std::vector<int> sts(parts.size(), RFR_OK);
        st = rfr_factor_batch(ctx, (int)parts.size(), ptrs.data(), degs.data(), res.data(), sts.data());
        if (st == RFR_OK)
            for (size_t i = 0; i < parts.size() && st == RFR_OK; ++i) {
                if (sts[i] != RFR_OK) { st = sts[i]; break; }
                size_t o = 0;
                for (int j = 0; j < res[i].n_factors; ++j) {
                    const int e = res[i].degrees[j];
                    PolyZ g(res[i].coeffs + o, res[i].coeffs + o + e + 1);
                    o += e + 1;
                    PolyZ h;
                    if (!back_transform(g, parts[i].f.back(), &h)) { st = RFR_E_OVERFLOW; break; }
                    fs.push_back({h, parts[i].mult});
                }
            }
        for (auto& r : res) rfr_factors_free(&r);
        if (st != RFR_OK) return st;
    }
    if (!product_check(fs, content, coeffs, degree)) return RFR_E_INTERNAL;
    return fill(fs, content, out);
}
