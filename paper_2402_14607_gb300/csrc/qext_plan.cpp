// Host-side plan construction: block factorisation, error bound and field
// polynomial (Algorithm 1's parameter line, Theorem 3.1, Sec. 3.2's GF(2^q)).
// Touches no GPU, so it runs (and is tested) on machines without one.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <new>

#include "qext_internal.h"

namespace {

// Polynomials over F_2 of degree < 64*kWords, as little-endian word arrays.
constexpr int kWords = 9;  // room for products of two degree-256 polynomials

struct BitPoly {
    uint64_t w[kWords];
    BitPoly() { std::memset(w, 0, sizeof w); }
    void flip(int d) { w[d >> 6] ^= uint64_t(1) << (d & 63); }
    bool get(int d) const { return (w[d >> 6] >> (d & 63)) & 1u; }
    int degree() const {
        for (int i = kWords - 1; i >= 0; --i)
            if (w[i]) return i * 64 + 63 - __builtin_clzll(w[i]);
        return -1;
    }
    bool is_one() const {
        if (w[0] != 1) return false;
        for (int i = 1; i < kWords; ++i)
            if (w[i]) return false;
        return true;
    }
    // this ^= other << s  (s >= 0, result must fit)
    void xor_shifted(const BitPoly &o, int s) {
        int ws = s >> 6, bs = s & 63;
        for (int i = kWords - 1; i >= ws; --i) {
            uint64_t v = o.w[i - ws] << bs;
            if (bs && i - ws - 1 >= 0) v |= o.w[i - ws - 1] >> (64 - bs);
            w[i] ^= v;
        }
    }
};

// a mod m by long division from the top coefficient down.
BitPoly poly_mod(BitPoly a, const BitPoly &m) {
    const int dm = m.degree();
    for (int d = a.degree(); d >= dm; d = a.degree()) a.xor_shifted(m, d - dm);
    return a;
}

// (a * a) mod m: squaring over F_2 spreads bit i to bit 2i.
BitPoly square_mod(const BitPoly &a, const BitPoly &m) {
    BitPoly s;
    for (int d = a.degree(); d >= 0; --d)
        if (a.get(d)) s.flip(2 * d);
    return poly_mod(s, m);
}

BitPoly poly_gcd(BitPoly a, BitPoly b) {
    while (b.degree() >= 0) {
        BitPoly r = poly_mod(a, b);
        a = b;
        b = r;
    }
    return a;
}

// Ben-Or's test: a degree-q polynomial P is irreducible iff
// gcd(P, x^(2^i) - x) = 1 for every i = 1 .. floor(q/2).
bool ben_or_irreducible(const BitPoly &P, int q) {
    if (P.degree() != q) return false;
    if (q == 1) return true;
    BitPoly u;  // u = x^(2^i) mod P
    u.flip(1);
    for (int i = 1; i <= q / 2; ++i) {
        u = square_mod(u, P);
        BitPoly t = u;
        t.flip(1);  // x^(2^i) - x
        if (t.degree() < 0) return false;  // P divides x^(2^i) - x with i < q
        if (!poly_gcd(P, t).is_one()) return false;
    }
    return true;
}

BitPoly make_poly(int q, const int *exps, int nexp) {
    BitPoly p;
    p.flip(q);
    for (int i = 0; i < nexp; ++i) p.flip(exps[i]);
    p.flip(0);
    return p;
}

// Minimum-weight irreducible polynomial, first in the order: trinomials
// x^q + x^a + 1 by a; then pentanomials x^q + x^c + x^b + x^a + 1 by c, b, a.
// Writes taps (descending, ending with the constant term's exponent 0).
bool choose_field_poly(int q, uint32_t *taps, uint32_t *ntaps) {
    if (q == 1) {  // F_2 itself: P = x, no reduction ever needed
        *ntaps = 0;
        return true;
    }
    for (int a = 1; a < q; ++a) {
        const int e[1] = {a};
        if (ben_or_irreducible(make_poly(q, e, 1), q)) {
            taps[0] = uint32_t(a);
            taps[1] = 0;
            *ntaps = 2;
            return true;
        }
    }
    for (int c = 3; c < q; ++c)
        for (int b = 2; b < c; ++b)
            for (int a = 1; a < b; ++a) {
                const int e[3] = {c, b, a};
                if (ben_or_irreducible(make_poly(q, e, 3), q)) {
                    taps[0] = uint32_t(c);
                    taps[1] = uint32_t(b);
                    taps[2] = uint32_t(a);
                    taps[3] = 0;
                    *ntaps = 4;
                    return true;
                }
            }
    return false;
}

// Theorem 3.1 for an n-bit block with min-entropy k (delta*q*n_p = k):
// log2 eps_blk = log2 sqrt(3) - 1/4 - (k/4 - n/8) + 2q.
double theorem31_log2_eps(uint32_t n, double k, uint32_t q) {
    return 0.5 * std::log2(3.0) - 0.25 - (k / 4.0 - double(n) / 8.0) + 2.0 * double(q);
}

constexpr int kMaxQ = 256;

}  // namespace

namespace qext {

bool gpu_q_supported(uint32_t q) {
    return q == 1 || q == 2 || q == 4 || q == 8 || q == 16 || q == 32 || q == 64;
}

bool field_poly(uint32_t q, uint32_t taps[4], uint32_t *ntaps) {
    return q >= 1 && q <= uint32_t(kMaxQ) && choose_field_poly(int(q), taps, ntaps);
}

double log2_eps_block(uint32_t n, double k, uint32_t q) { return theorem31_log2_eps(n, k, q); }

uint32_t max_field_degree() { return uint32_t(kMaxQ); }

}  // namespace qext

extern "C" {

const char *qext_status_string(int status) {
    switch (status) {
        case QEXT_OK: return "QEXT_OK";
        case QEXT_E_INVAL: return "QEXT_E_INVAL: invalid argument";
        case QEXT_E_ENTROPY: return "QEXT_E_ENTROPY: min-entropy rate must exceed 1/2";
        case QEXT_E_PARAM: return "QEXT_E_PARAM: no block factorisation meets eps and m";
        case QEXT_E_UNSUPPORTED: return "QEXT_E_UNSUPPORTED: no GPU kernel for this field size";
        case QEXT_E_CUDA: return "QEXT_E_CUDA: CUDA runtime error";
        case QEXT_E_TIMEOUT: return "QEXT_E_TIMEOUT: a kernel gave up a bounded wait";
        case QEXT_E_BUDGET: return "QEXT_E_BUDGET: device memory budget exhausted";
        case QEXT_E_STATE: return "QEXT_E_STATE: call not allowed in the object's state";
        case QEXT_E_NOSPACE: return "QEXT_E_NOSPACE: output buffer too small";
        case QEXT_E_LIMIT: return "QEXT_E_LIMIT: request exceeds a fixed capacity";
        default: return "QEXT_E_UNKNOWN";
    }
}

int qext_plan_create(uint32_t n, uint32_t m, double k, double eps, qext_plan **out) {
    if (!out) return QEXT_E_INVAL;
    *out = nullptr;
    if (n == 0 || !(k > 0.0) || k > double(n) || !(eps > 0.0) || !(eps < 1.0))
        return QEXT_E_INVAL;
    const double gap = 2.0 * k - double(n);  // (2 delta - 1) * n
    if (!(gap > 0.0)) return QEXT_E_ENTROPY;
    // n_min = ceil(24 / (2 delta - 1)) = least d with d * (2k - n) >= 24 n
    uint64_t dmin = uint64_t(std::floor(24.0 * double(n) / gap));
    if (dmin < 1) dmin = 1;
    while (dmin > 1 && double(dmin - 1) * gap >= 24.0 * double(n)) --dmin;
    while (double(dmin) * gap < 24.0 * double(n)) ++dmin;
    const double log2_target = std::log2(eps);
    for (uint64_t d = dmin; d <= n; ++d) {
        if (n % d) continue;
        const uint32_t q = uint32_t(n / d);
        if (m && m > q) break;  // q only shrinks from here on
        const double l2 = theorem31_log2_eps(n, k, q);
        if (l2 > log2_target) continue;
        if (q > uint32_t(kMaxQ)) continue;
        qext_plan *p = new (std::nothrow) qext_plan();
        if (!p) return QEXT_E_INVAL;
        p->n = n;
        p->n_p = uint32_t(d);
        p->q = q;
        p->m = m ? m : q;
        p->k = k;
        p->eps = eps;
        p->log2_eps = l2;
        if (!choose_field_poly(int(q), p->taps, &p->ntaps)) {
            delete p;
            return QEXT_E_PARAM;
        }
        // two reduction folds suffice when the top tap c satisfies 2c - 2 < q
        p->gpu_supported = qext::gpu_q_supported(q) && n % 32 == 0 && (p->ntaps == 0 || 2 * p->taps[0] < q + 2);
        p->gpu_q80 = q == 80 && 2 * p->taps[0] < q + 2;
        *out = p;
        return QEXT_OK;
    }
    return QEXT_E_PARAM;
}

int qext_destroy(qext_plan *p) {
    delete p;
    return QEXT_OK;
}

int qext_plan_info(const qext_plan *p, uint32_t *q, uint32_t *n_p, uint32_t *m, double *log2_eps_block,
                   uint64_t poly_taps[4], int *gpu_supported) {
    if (!p) return QEXT_E_INVAL;
    if (q) *q = p->q;
    if (n_p) *n_p = p->n_p;
    if (m) *m = p->m;
    if (log2_eps_block) *log2_eps_block = p->log2_eps;
    if (poly_taps) {
        for (int i = 0; i < 4; ++i) poly_taps[i] = 0;
        int o = 0;
        for (uint32_t i = 0; i < p->ntaps; ++i)
            if (p->taps[i]) poly_taps[o++] = p->taps[i];
    }
    if (gpu_supported) *gpu_supported = p->gpu_supported ? 1 : p->gpu_q80 ? 2 : 0;
    return QEXT_OK;
}

int qext_alg1_params(double N_samples, uint32_t b, double delta, double eps, uint32_t *n_p, uint32_t *q) {
    if (!n_p || !q || !(N_samples > 0.0) || b == 0 || !(eps > 0.0) || !(eps < 1.0)) return QEXT_E_INVAL;
    if (!(delta > 0.5) || !(delta <= 1.0)) return delta > 1.0 ? QEXT_E_INVAL : QEXT_E_ENTROPY;
    const double np_ = std::ceil(24.0 / (2.0 * delta - 1.0));
    const double qq = double(b) * std::ceil(std::log2(N_samples / (eps * np_)) / double(b));
    if (!(qq >= 1.0) || qq > 4294967295.0) return QEXT_E_INVAL;
    *n_p = uint32_t(np_);
    *q = uint32_t(qq);
    return QEXT_OK;
}

}  // extern "C"
