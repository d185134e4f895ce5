// Host-side plan construction: block factorisation, error bound and field
// polynomial (Algorithm 1's parameter line, Theorem 3.1, Sec. 3.2's GF(2^q)).
// Touches no GPU, so it runs (and is tested) on machines without one.
#include <cmath>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "qext_internal.h"

namespace {

constexpr int kMaxQ = 2048;  // largest field degree (Algorithm 2's fields up to its 128th block at q_1 = Delta b = 16)

// Polynomials over F_2 as little-endian arrays of 64-bit words; kPW words
// hold a square (degree <= 2 kMaxQ - 2) before reduction.
constexpr int kPW = 2 * kMaxQ / 64 + 2;

struct Poly {
    uint64_t w[kPW];
    Poly() { std::memset(w, 0, sizeof w); }
    void flip(int d) { w[d >> 6] ^= uint64_t(1) << (d & 63); }
    bool get(int d) const { return (w[d >> 6] >> (d & 63)) & 1u; }
    int degree() const {
        for (int i = kPW - 1; i >= 0; --i)
            if (w[i]) return i * 64 + 63 - __builtin_clzll(w[i]);
        return -1;
    }
    // this ^= o * x^s (the shifted copy must fit)
    void xor_shifted(const Poly &o, int s) {
        const int ws = s >> 6, bs = s & 63;
        for (int i = kPW - 1; i >= ws; --i) {
            uint64_t v = o.w[i - ws] << bs;
            if (bs && i - ws - 1 >= 0) v |= o.w[i - ws - 1] >> (64 - bs);
            w[i] ^= v;
        }
    }
};

// A candidate field polynomial P = x^q + sum_t x^e[t] (e[] includes 0).
struct Sparse {
    int q;
    int ne;
    int e[4];
    Poly dense() const {
        Poly p;
        p.flip(q);
        for (int t = 0; t < ne; ++t) p.flip(e[t]);
        return p;
    }
};

// Squaring over F_2 spreads bit i to bit 2i: one table lookup per byte.
struct SpreadTable {
    uint16_t t[256];
    SpreadTable() {
        for (int v = 0; v < 256; ++v) {
            uint16_t r = 0;
            for (int i = 0; i < 8; ++i)
                if (v & (1 << i)) r |= uint16_t(1u << (2 * i));
            t[v] = r;
        }
    }
};
const SpreadTable kSpread;

// r = a^2 (a has nw words, r gets 2 nw words; the rest of r is not touched)
void square_words(const uint64_t *a, int nw, uint64_t *r) {
    for (int i = 0; i < nw; ++i) {
        uint64_t lo = 0, hi = 0;
        for (int k = 0; k < 4; ++k) {
            lo |= uint64_t(kSpread.t[(a[i] >> (8 * k)) & 0xFF]) << (16 * k);
            hi |= uint64_t(kSpread.t[(a[i] >> (32 + 8 * k)) & 0xFF]) << (16 * k);
        }
        r[2 * i] = lo;
        r[2 * i + 1] = hi;
    }
}

// r mod P in place for a sparse P, by whole-word folds: with H = the part of
// r at and above x^q, r = (r mod x^q) + H * (P - x^q), repeated until nothing
// remains at or above x^q.  r has nw words.
void reduce_sparse(uint64_t *r, int nw, const Sparse &P) {
    const int q = P.q, qw = q >> 6, qb = q & 63;
    uint64_t H[kPW];
    for (;;) {
        bool any = false;
        const int hn = nw - qw;
        for (int i = 0; i < hn; ++i) {
            uint64_t v = r[qw + i] >> qb;
            if (qb && qw + i + 1 < nw) v |= r[qw + i + 1] << (64 - qb);
            H[i] = v;
            any |= v != 0;
        }
        if (!any) return;
        if (qb) r[qw] &= (uint64_t(1) << qb) - 1;
        for (int i = (qb ? qw + 1 : qw); i < nw; ++i) r[i] = 0;
        for (int t = 0; t < P.ne; ++t) {
            const int s = P.e[t], ws = s >> 6, bs = s & 63;
            for (int i = hn - 1; i >= 0; --i) {
                if (!H[i]) continue;
                const int d = i + ws;
                if (d < nw) r[d] ^= H[i] << bs;
                if (bs && d + 1 < nw) r[d + 1] ^= H[i] >> (64 - bs);
            }
        }
    }
}

// a mod m by long division (dense m), for the gcds of Rabin's test.
Poly poly_mod(Poly a, const Poly &m) {
    const int dm = m.degree();
    for (int d = a.degree(); d >= dm; d = a.degree()) a.xor_shifted(m, d - dm);
    return a;
}

Poly poly_gcd(Poly a, Poly b) {
    while (b.degree() >= 0) {
        Poly r = poly_mod(a, b);
        a = b;
        b = r;
    }
    return a;
}

// Small irreducible polynomials f (degrees 2..8, bit masks), found by trial
// division among themselves, with the powers x^k mod f for k < 2^deg(f) - 1:
// x^(2^d - 1) = 1 mod f for an irreducible f of degree d other than x, so
// x^e mod f = x^(e mod (2^d - 1)) mod f.
struct SmallIrreducibles {
    static constexpr int kMax = 80;
    int n = 0;
    uint32_t f[kMax];
    uint32_t period[kMax];
    uint16_t pw[kMax][255];
    static int deg(uint32_t a) { return a ? 31 - __builtin_clz(a) : -1; }
    static uint32_t mod_small(uint32_t a, uint32_t m) {
        const int dm = deg(m);
        for (int d = deg(a); d >= dm; d = deg(a)) a ^= m << (d - dm);
        return a;
    }
    SmallIrreducibles() {
        for (uint32_t m = 4; m < 512 && n < kMax; ++m) {      // degrees 2 .. 8
            bool irr = (m & 1u) && mod_small(m, 3u) != 0;    // no factor x or x + 1
            for (int i = 0; i < n && irr; ++i)
                if (mod_small(m, f[i]) == 0) irr = false;
            if (!irr) continue;
            f[n] = m;
            period[n] = (1u << deg(m)) - 1u;
            uint32_t v = 1;
            for (uint32_t k = 0; k < period[n]; ++k) {
                pw[n][k] = uint16_t(v);
                v = mod_small(v << 1, m);
            }
            ++n;
        }
    }
};
const SmallIrreducibles kSmall;

// A factor of degree <= 8, by trial division: P mod f = sum of x^e mod f
// over P's terms.  (Candidates have an odd number of terms and a constant
// term, so neither x nor x + 1 divides them.)
bool has_small_factor(const Sparse &P) {
    if (P.q <= 8) return false;
    for (int i = 0; i < kSmall.n; ++i) {
        const uint32_t per = kSmall.period[i];
        uint32_t r = kSmall.pw[i][uint32_t(P.q) % per];
        for (int t = 0; t < P.ne; ++t) r ^= kSmall.pw[i][uint32_t(P.e[t]) % per];
        if (r == 0) return true;
    }
    return false;
}

// Rabin's test: P of degree q is irreducible iff x^(2^q) = x mod P and
// gcd(x^(2^(q/r)) - x, P) = 1 for every prime r dividing q.  The powers
// x^(2^k) come from q squarings with sparse folds.
bool rabin_irreducible(const Sparse &P) {
    const int q = P.q;
    if (q == 1) return true;
    int primes[16], np = 0, rem = q;
    for (int r = 2; r <= rem; ++r)
        if (rem % r == 0) {
            primes[np++] = r;
            while (rem % r == 0) rem /= r;
        }
    const int nw = q / 64 + 1, sw = 2 * nw;
    uint64_t u[kPW] = {0}, t[kPW];
    u[0] = 2;  // x
    Poly saved[16];
    for (int k = 1; k <= q; ++k) {
        std::memset(t, 0, sizeof(uint64_t) * sw);
        square_words(u, nw, t);
        reduce_sparse(t, sw, P);
        std::memcpy(u, t, sizeof(uint64_t) * nw);
        for (int i = 0; i < np; ++i)
            if (k == q / primes[i]) std::memcpy(saved[i].w, u, sizeof(uint64_t) * nw);
    }
    if (u[0] != 2) return false;
    for (int i = 1; i < nw; ++i)
        if (u[i]) return false;
    const Poly dense = P.dense();
    for (int i = 0; i < np; ++i) {
        Poly v = saved[i];
        v.flip(1);  // x^(2^(q/r)) - x
        if (v.degree() < 0) return false;
        if (poly_gcd(dense, v).degree() != 0) return false;
    }
    return true;
}

bool irreducible(const Sparse &P) { return !has_small_factor(P) && rabin_irreducible(P); }

// Minimum-weight irreducible polynomial, first in the order: trinomials
// x^q + x^a + 1 by a; then pentanomials x^q + x^c + x^b + x^a + 1 by c, b, a.
// Writes taps (descending, ending with the constant term's exponent 0).
bool search_field_poly(int q, uint32_t *taps, uint32_t *ntaps) {
    if (q == 1) {  // F_2 itself: P = x, no reduction ever needed
        *ntaps = 0;
        return true;
    }
    for (int a = 1; a < q; ++a) {
        const Sparse P{q, 2, {a, 0, 0, 0}};
        if (irreducible(P)) {
            taps[0] = uint32_t(a);
            taps[1] = 0;
            *ntaps = 2;
            return true;
        }
    }
    for (int c = 3; c < q; ++c)
        for (int b = 2; b < c; ++b)
            for (int a = 1; a < b; ++a) {
                const Sparse P{q, 4, {c, b, a, 0}};
                if (irreducible(P)) {
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

// The search's result per degree, kept for the process (a search at the
// largest degrees takes a large fraction of a second).
struct FieldCache {
    std::mutex mu;
    bool known[kMaxQ + 1] = {};
    uint32_t taps[kMaxQ + 1][4];
    uint32_t ntaps[kMaxQ + 1];
};
FieldCache g_fields;

bool choose_field_poly(int q, uint32_t *taps, uint32_t *ntaps) {
    if (q < 1 || q > kMaxQ) return false;
    {
        std::lock_guard<std::mutex> lock(g_fields.mu);
        if (g_fields.known[q]) {
            std::memcpy(taps, g_fields.taps[q], sizeof(uint32_t) * 4);
            *ntaps = g_fields.ntaps[q];
            return true;
        }
    }
    uint32_t t[4] = {0, 0, 0, 0}, nt = 0;
    if (!search_field_poly(q, t, &nt)) return false;
    std::lock_guard<std::mutex> lock(g_fields.mu);
    std::memcpy(g_fields.taps[q], t, sizeof t);
    g_fields.ntaps[q] = nt;
    g_fields.known[q] = true;
    std::memcpy(taps, t, sizeof t);
    *ntaps = nt;
    return true;
}

// Theorem 3.1 for an n-bit block with min-entropy k (delta*q*n_p = k):
// log2 eps_blk = log2 sqrt(3) - 1/4 - (k/4 - n/8) + 2q.
double theorem31_log2_eps(uint32_t n, double k, uint32_t q) {
    return 0.5 * std::log2(3.0) - 0.25 - (k / 4.0 - double(n) / 8.0) + 2.0 * double(q);
}


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
