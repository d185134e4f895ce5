/*
 * qext_oracle.c -- plain, slow, obviously correct CPU oracle for the block-wise
 * two-source extractor Ext_bs^eq (Algorithm 1) of Li & Zhou, "Real-Time
 * Seedless Post-Processing for Quantum Random Number Generators"
 * (arXiv 2402.14607).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the reference the CUDA path is
 * checked against.  Only the tests, the smoke check and the benchmark's CPU
 * baseline may load it.  It shares no code, header, table or constant with the
 * CUDA library: it has its own polynomial arithmetic, its own irreducibility
 * test and its own bit addressing, written for clarity, not speed.
 *
 * Conventions (the paper fixes none of these; they are the readings this
 * project adopts, and every function below follows them):
 *   - A stream is a little-endian array of uint32 words; stream bit t is bit
 *     (t mod 32) of word floor(t/32).  An ADC sample s of b bits occupies
 *     stream bits [s*b, (s+1)*b), least significant bit first.
 *   - Block l (0-based) of a source is stream bits [l*n, (l+1)*n), n = q*n_p.
 *     Element i (0-based) of the block is bits [l*n + i*q, l*n + (i+1)*q);
 *     element bit j is the coefficient of alpha^j (polynomial basis).
 *   - GF(2^q) = F_2[alpha] / P(alpha).  P is given to every routine as a full
 *     coefficient vector (bit d of the vector = coefficient of x^d, degree q).
 *   - Output: Z^(l) truncated to its first m coefficients (alpha^0..alpha^m-1)
 *     occupies output bits [l*m, (l+1)*m); unused bits of the last word are 0.
 *
 * Field elements and polynomials are arrays of uint64 words, least
 * significant word first, holding up to ORC_MAXQ coefficients.
 */
#include <stdint.h>
#include <stdlib.h>
#include <string.h>
#include <math.h>
#ifdef _OPENMP
#include <omp.h>
#endif

#define ORC_MAXQ 2048                     /* largest field degree supported   */
#define ORC_W ((ORC_MAXQ + 64) / 64 + 1)  /* words of a degree <= MAXQ poly   */
#define ORC_W2 (2 * ORC_W)                /* words of a product before mod    */

/* ------------------------------------------------------------------------ */
/* Bit helpers on word arrays (uint64 polynomial coefficient vectors).       */
/* ------------------------------------------------------------------------ */
static int pbit(const uint64_t *a, int d) { return (int)((a[d >> 6] >> (d & 63)) & 1u); }
static void pset(uint64_t *a, int d) { a[d >> 6] |= (uint64_t)1 << (d & 63); }
static void pflip(uint64_t *a, int d) { a[d >> 6] ^= (uint64_t)1 << (d & 63); }

/* degree of a polynomial stored in nw words; -1 for the zero polynomial */
static int pdeg(const uint64_t *a, int nw)
{
    for (int w = nw - 1; w >= 0; --w)
        if (a[w]) {
            int d = 63;
            while (!((a[w] >> d) & 1u)) --d;
            return w * 64 + d;
        }
    return -1;
}

/* ------------------------------------------------------------------------ */
/* GF(2^q) multiplication, bit-serial (Sec. 3.2, the field F_{2^q} with      */
/* addition = bitwise parity).  Right-to-left shift-and-add: for each bit j  */
/* of b, add alpha^j * a when that bit is set, where alpha^j * a is kept     */
/* reduced mod P after every single shift by alpha.                          */
/* ------------------------------------------------------------------------ */
void orc_gf_mul(int q, const uint64_t *poly, const uint64_t *a, const uint64_t *b, uint64_t *out)
{
    uint64_t sh[ORC_W], acc[ORC_W];
    int nw = q / 64 + 1;
    int pe[ORC_MAXQ + 1], npe = 0;                    /* exponents of P's nonzero terms */
    for (int d = 0; d <= q; ++d)
        if (pbit(poly, d)) pe[npe++] = d;
    memset(sh, 0, sizeof sh);
    memset(acc, 0, sizeof acc);
    for (int d = 0; d < q; ++d)
        if (pbit(a, d)) pset(sh, d);                  /* sh = a (reduced input) */
    for (int j = 0; j < q; ++j) {
        if (pbit(b, j))
            for (int w = 0; w < nw; ++w) acc[w] ^= sh[w];   /* acc += alpha^j a  */
        /* sh = sh * alpha mod P: shift by one, subtract P if degree reached q */
        for (int w = nw - 1; w > 0; --w) sh[w] = (sh[w] << 1) | (sh[w - 1] >> 63);
        sh[0] <<= 1;
        if (pbit(sh, q))
            for (int t = 0; t < npe; ++t) pflip(sh, pe[t]);   /* sh -= P */
    }
    int ow = (q + 63) / 64;
    for (int w = 0; w < ow; ++w) out[w] = acc[w];
}

/* ------------------------------------------------------------------------ */
/* Polynomial arithmetic over F_2 used only by the irreducibility test.      */
/* ------------------------------------------------------------------------ */

/* r ^= m * x^s (word arrays of ORC_W2 words; the shifted copy must fit) */
static void pxor_shifted(uint64_t *r, const uint64_t *m, int s)
{
    int ws = s >> 6, bs = s & 63;
    for (int i = ORC_W2 - 1; i >= ws; --i) {
        uint64_t v = m[i - ws] << bs;
        if (bs && i - ws - 1 >= 0) v |= m[i - ws - 1] >> (64 - bs);
        r[i] ^= v;
    }
}

/*
 * r = a mod m (m nonzero); all arrays ORC_W2 words.  Long division from the
 * top coefficient down: each set coefficient d >= deg m of the running
 * remainder is cleared by subtracting m * x^(d - deg m).  A sparse m (at most
 * 8 terms, e.g. a field polynomial) is subtracted term by term, a dense one
 * as a shifted word copy; both are the same subtraction.
 */
static void pmod(const uint64_t *a, const uint64_t *m, uint64_t *r)
{
    int dm = pdeg(m, ORC_W2);
    int me[8], nme = 0, sparse = 1;
    for (int e = 0; e <= dm; ++e)
        if (pbit(m, e)) {
            if (nme == 8) { sparse = 0; break; }
            me[nme++] = e;
        }
    memcpy(r, a, sizeof(uint64_t) * ORC_W2);
    for (int d = pdeg(r, ORC_W2); d >= dm; --d)
        if (pbit(r, d)) {
            if (sparse)
                for (int t = 0; t < nme; ++t) pflip(r, d - dm + me[t]);
            else
                pxor_shifted(r, m, d - dm);
        }
}

/* r = a^2 mod m: over F_2, (sum a_i x^i)^2 = sum a_i x^(2i) */
static void psqrmod(const uint64_t *a, const uint64_t *m, uint64_t *r)
{
    uint64_t sq[ORC_W2];
    memset(sq, 0, sizeof sq);
    int da = pdeg(a, ORC_W2);
    for (int i = 0; i <= da; ++i)
        if (pbit(a, i)) pset(sq, 2 * i);
    pmod(sq, m, r);
}

/* g = gcd(a, b), Euclid */
static void pgcd(const uint64_t *a, const uint64_t *b, uint64_t *g)
{
    uint64_t u[ORC_W2], v[ORC_W2], t[ORC_W2];
    memcpy(u, a, sizeof u);
    memcpy(v, b, sizeof v);
    while (pdeg(v, ORC_W2) >= 0) {
        pmod(u, v, t);
        memcpy(u, v, sizeof u);
        memcpy(v, t, sizeof v);
    }
    memcpy(g, u, sizeof u);
}

/* r = x^(2^e) mod m by e repeated squarings of x */
static void x_pow_2e(int e, const uint64_t *m, uint64_t *r)
{
    uint64_t x[ORC_W2], t[ORC_W2];
    memset(x, 0, sizeof x);
    pset(x, 1);
    pmod(x, m, r);
    for (int i = 0; i < e; ++i) {
        psqrmod(r, m, t);
        memcpy(r, t, sizeof t);
    }
}

/*
 * Rabin's irreducibility test for a degree-q polynomial over F_2:
 * P is irreducible iff x^(2^q) = x (mod P) and, for every prime r dividing q,
 * gcd(x^(2^(q/r)) - x mod P, P) = 1.
 * Returns 1 if irreducible, 0 otherwise.
 */
int orc_is_irreducible(int q, const uint64_t *poly)
{
    uint64_t m[ORC_W2], r[ORC_W2], g[ORC_W2];
    if (q < 1 || q > ORC_MAXQ) return 0;
    memset(m, 0, sizeof m);
    for (int d = 0; d <= q; ++d)
        if (pbit(poly, d)) pset(m, d);
    if (pdeg(m, ORC_W2) != q) return 0;
    if (q == 1) return 1;
    x_pow_2e(q, m, r);
    pflip(r, 1);                                   /* r = x^(2^q) - x mod P */
    if (pdeg(r, ORC_W2) >= 0) return 0;
    int rem = q;
    for (int p = 2; p <= rem; ++p) {
        if (rem % p) continue;
        while (rem % p == 0) rem /= p;
        x_pow_2e(q / p, m, r);
        pflip(r, 1);
        pgcd(m, r, g);
        if (pdeg(g, ORC_W2) != 0) return 0;
    }
    return 1;
}

/*
 * Field polynomial choice (the paper leaves P_q open, Sec. 3.2): the
 * lexicographically first irreducible polynomial of minimum weight.
 *   q = 1: F_2 itself, P = x (multiplication is AND).
 *   else a trinomial x^q + x^a + 1 with the smallest a, if one exists;
 *   else a pentanomial x^q + x^c + x^b + x^a + 1, q > c > b > a >= 1,
 *   minimising c, then b, then a.
 * Writes the coefficient vector to poly (q/64+1 words) and the taps below q
 * (descending, the constant term excluded) to taps[0..2] (unused = 0).
 * Returns the weight (2, 3 or 5), or 0 if none was found.
 */
int orc_select_poly(int q, uint64_t *poly, int *taps)
{
    int nw = q / 64 + 1;
    taps[0] = taps[1] = taps[2] = 0;
    if (q < 1 || q > ORC_MAXQ) return 0;
    if (q == 1) {
        memset(poly, 0, sizeof(uint64_t) * nw);
        pset(poly, 1);
        return 2;
    }
    /* trinomials x^q + x^a + 1 in the order of a; the candidates are tested in
       parallel and the smallest irreducible one is taken */
    int best = q;
#pragma omp parallel for schedule(dynamic, 1) reduction(min:best)
    for (int a = 1; a < q; ++a) {
        if (a >= best) continue;
        uint64_t p[ORC_W];
        memset(p, 0, sizeof p);
        pset(p, q); pset(p, a); pset(p, 0);
        if (orc_is_irreducible(q, p)) best = a;
    }
    if (best < q) {
        memset(poly, 0, sizeof(uint64_t) * nw);
        pset(poly, q); pset(poly, best); pset(poly, 0);
        taps[0] = best;
        return 3;
    }
    /* pentanomials x^q + x^c + x^b + x^a + 1, q > c > b > a >= 1, in the order
       of c, then b, then a: the candidates with one c are tested together */
    for (int c = 3; c < q; ++c) {
        int n = (c - 1) * (c - 2) / 2, first = n;   /* pairs (b, a), b > a >= 1, in order */
#pragma omp parallel for schedule(dynamic, 1) reduction(min:first)
        for (int k = 0; k < n; ++k) {
            if (k >= first) continue;
            int b = 2, left = k;                    /* the k-th pair in the (b, a) order */
            while (left >= b - 1) { left -= b - 1; ++b; }
            int a = 1 + left;
            uint64_t p[ORC_W];
            memset(p, 0, sizeof p);
            pset(p, q); pset(p, c); pset(p, b); pset(p, a); pset(p, 0);
            if (orc_is_irreducible(q, p)) first = k;
        }
        if (first < n) {
            int b = 2, left = first;
            while (left >= b - 1) { left -= b - 1; ++b; }
            int a = 1 + left;
            memset(poly, 0, sizeof(uint64_t) * nw);
            pset(poly, q); pset(poly, c); pset(poly, b); pset(poly, a); pset(poly, 0);
            taps[0] = c; taps[1] = b; taps[2] = a;
            return 5;
        }
    }
    return 0;
}

/* ------------------------------------------------------------------------ */
/* Inner-product extractor, Definition 3.2:                                  */
/*   Ext_IP^{n,q}(x, y) = sum_{i=1..n} x_i * y_i   in GF(2^q).               */
/* xs, ys: n_p elements, each (q+63)/64 words; out: (q+63)/64 words.         */
/* ------------------------------------------------------------------------ */
void orc_ext_ip(int q, int n_p, const uint64_t *poly, const uint64_t *xs, const uint64_t *ys, uint64_t *out)
{
    int ew = (q + 63) / 64;
    uint64_t prod[ORC_W];
    memset(out, 0, sizeof(uint64_t) * ew);
    for (int i = 0; i < n_p; ++i) {
        orc_gf_mul(q, poly, xs + (size_t)i * ew, ys + (size_t)i * ew, prod);
        for (int w = 0; w < ew; ++w) out[w] ^= prod[w];   /* +_q is bitwise parity */
    }
}

/* stream bit t of a word array */
static int sbit(const uint32_t *s, uint64_t t) { return (int)((s[t >> 5] >> (t & 31)) & 1u); }

/*
 * Algorithm 1 (Ext_bs^eq) over nblocks whole blocks of two packed streams.
 * For l = 1..nblocks: I_l is the next q*n_p stream bits of each source
 * (consecutive, non-overlapping windows: the cursor advances by one block),
 * Z^(l) = Ext_IP^{n_p,q}(X_{I_l}, Y_{I_l}), and Z^(l) is output in order,
 * truncated to its first m bits.  out must hold ceil(nblocks*m/32) words and
 * is fully overwritten.  threads <= 0 means all processors (OpenMP builds).
 * Returns 0, or -1 on bad arguments.
 */
int orc_extract(int q, int n_p, int m, const uint64_t *poly, const uint32_t *x, const uint32_t *y,
                uint64_t nblocks, uint32_t *out, int threads)
{
    if (q < 1 || q > ORC_MAXQ || n_p < 1 || m < 1 || m > q) return -1;
    uint64_t n = (uint64_t)q * (uint64_t)n_p;
    uint64_t outw = (nblocks * (uint64_t)m + 31) / 32;
    memset(out, 0, sizeof(uint32_t) * outw);
    int ew = (q + 63) / 64;
    (void)threads;
#ifdef _OPENMP
    int nthreads = threads > 0 ? threads : omp_get_num_procs();
#pragma omp parallel num_threads(nthreads)
#endif
    {
        uint64_t *xs = (uint64_t *)calloc((size_t)n_p * ew, sizeof(uint64_t));
        uint64_t *ys = (uint64_t *)calloc((size_t)n_p * ew, sizeof(uint64_t));
        uint64_t z[ORC_W];
#ifdef _OPENMP
#pragma omp for schedule(static)
#endif
        for (int64_t l = 0; l < (int64_t)nblocks; ++l) {
            uint64_t base = (uint64_t)l * n;                     /* I_l starts here */
            memset(xs, 0, sizeof(uint64_t) * (size_t)n_p * ew);
            memset(ys, 0, sizeof(uint64_t) * (size_t)n_p * ew);
            for (int i = 0; i < n_p; ++i)
                for (int j = 0; j < q; ++j) {
                    uint64_t t = base + (uint64_t)i * q + j;
                    if (sbit(x, t)) pset(xs + (size_t)i * ew, j);
                    if (sbit(y, t)) pset(ys + (size_t)i * ew, j);
                }
            orc_ext_ip(q, n_p, poly, xs, ys, z);                   /* Z^(l) */
            for (int j = 0; j < m; ++j)                              /* first m bits */
                if (pbit(z, j)) {
                    uint64_t o = (uint64_t)l * m + j;
                    /* blocks write disjoint bit ranges; word sharing is guarded */
#ifdef _OPENMP
#pragma omp atomic
#endif
                    out[o >> 5] |= (uint32_t)1 << (o & 31);
                }
        }
        free(xs);
        free(ys);
    }
    return 0;
}

/*
 * Algorithm 2 (Ext_bs^neq, Sec. 3.3) over its first nblocks blocks.
 * Parameters q_1 = q1 and the step dq = Delta * b; n = n_p elements per
 * block.  Following the algorithm: the cursor i starts at the first sample;
 * block l takes the window I_l = [i, i - 1 + q_l n / b] of each source,
 * computes Z^(l) = Ext_IP^{n, q_l}(X_{I_l}, Y_{I_l}) in GF(2^{q_l}) (with
 * that degree's field polynomial, chosen as for Algorithm 1), outputs it, then
 * i := i + q_l n / b and q_{l+1} := q_l + Delta b.  In stream bits the window
 * is the next q_l * n bits and the outputs are concatenated, q_l bits each.
 * out must hold ceil(sum q_l / 32) words and is fully overwritten.
 * Returns 0, or -1 on bad arguments (some q_l outside 1..ORC_MAXQ).
 */
int orc_extract_alg2(int n_p, int q1, int dq, int nblocks, const uint32_t *x, const uint32_t *y, uint32_t *out,
                     const int *given_taps)
{
    if (n_p < 1 || q1 < 1 || dq < 0 || nblocks < 0) return -1;
    if ((int64_t)q1 + (int64_t)dq * (nblocks > 0 ? nblocks - 1 : 0) > ORC_MAXQ) return -1;
    uint64_t total = 0;
    for (int l = 0; l < nblocks; ++l) total += (uint64_t)(q1 + l * dq);
    memset(out, 0, sizeof(uint32_t) * ((total + 31) / 32));
    uint64_t i = 0;   /* the cursor, in stream bits */
    uint64_t o = 0;   /* output bits so far */
    int ql = q1;      /* q_l */
    for (int l = 0; l < nblocks; ++l) {
        uint64_t poly[ORC_W], z[ORC_W];
        int taps[3];
        if (given_taps) {   /* P_{q_l} given as its taps (c, b, a; zero past a trinomial's) */
            memset(poly, 0, sizeof poly);
            pset(poly, ql); pset(poly, 0);
            for (int t = 0; t < 3; ++t)
                if (given_taps[3 * l + t]) pset(poly, given_taps[3 * l + t]);
        } else if (!orc_select_poly(ql, poly, taps)) {
            return -1;
        }
        int ew = (ql + 63) / 64;
        uint64_t *xs = (uint64_t *)calloc((size_t)n_p * ew, sizeof(uint64_t));
        uint64_t *ys = (uint64_t *)calloc((size_t)n_p * ew, sizeof(uint64_t));
        for (int e = 0; e < n_p; ++e)               /* X_{I_l}: n elements of q_l bits */
            for (int j = 0; j < ql; ++j) {
                uint64_t t = i + (uint64_t)e * ql + j;
                if (sbit(x, t)) pset(xs + (size_t)e * ew, j);
                if (sbit(y, t)) pset(ys + (size_t)e * ew, j);
            }
        orc_ext_ip(ql, n_p, poly, xs, ys, z);     /* Z^(l) */
        free(xs);
        free(ys);
        for (int j = 0; j < ql; ++j)                /* output Z^(l) */
            if (pbit(z, j)) out[(o + j) >> 5] |= (uint32_t)1 << ((o + j) & 31);
        i += (uint64_t)ql * (uint64_t)n_p;         /* i := i + q_l n / b (in bits: q_l n) */
        o += (uint64_t)ql;
        ql += dq;                                   /* q_{l+1} := q_l + Delta b */
    }
    return 0;
}

/*
 * log2 of Theorem 3.3's bound on the error of the first nblocks outputs of
 * Algorithm 2 (rate delta, n = n_p):
 *   sqrt(3) * sum_l 2^(-1/4 - (delta/4 - 1/8) q_l n + 2 q_l).
 */
double orc_alg2_log2_error(int n_p, double delta, int q1, int dq, int nblocks)
{
    double sum = 0.0;
    for (int l = 0; l < nblocks; ++l) {
        double ql = (double)(q1 + l * dq);
        sum += pow(2.0, -0.25 - (delta / 4.0 - 0.125) * ql * (double)n_p + 2.0 * ql);
    }
    return 0.5 * log2(3.0) + log2(sum);
}

/*
 * log2 of the per-block error of Theorem 3.1 for an n-bit block (n = q*n_p)
 * of min-entropy k bits (k = delta*q*n_p):
 *   eps_blk = sqrt(3) * 2^(-1/4 - (delta/4 - 1/8) q n_p + 2q)
 *   log2 eps_blk = log2(sqrt 3) - 1/4 - (k/4 - n/8) + 2q.
 */
double orc_log2_eps_block(uint32_t n, double k, uint32_t q)
{
    return 0.5 * log2(3.0) - 0.25 - (k / 4.0 - (double)n / 8.0) + 2.0 * (double)q;
}

/*
 * Per-block plan from Definition 2.3's (t, m, k, eps) with t = n:
 *   delta = k/n must exceed 1/2 (the construction needs rate > 1/2);
 *   n_min = ceil(24 / (2 delta - 1)) (Algorithm 1's n), evaluated exactly as
 *           the least integer d with d*(2k - n) >= 24n;
 *   candidates: divisors d of n with d >= n_min, increasing, q = n/d;
 *   pick the first with log2 eps_blk(q) <= log2 eps and (m == 0 or m <= q).
 * m == 0 selects m = q (the whole field element, Theorem 3.4's output length).
 * Returns 0 on success, -2 if delta <= 1/2, -3 if no candidate meets eps,
 * -1 on bad arguments.
 */
int orc_plan(uint32_t n, uint32_t m, double k, double eps, uint32_t *n_p, uint32_t *q, uint32_t *m_out,
             double *log2_eps)
{
    if (n == 0 || !(eps > 0.0) || !(eps < 1.0) || !(k > 0.0) || k > (double)n) return -1;
    double gap = 2.0 * k - (double)n;
    if (!(gap > 0.0)) return -2;
    uint64_t dmin = 1;
    while ((double)dmin * gap < 24.0 * (double)n) ++dmin;
    double le = log2(eps);
    for (uint64_t d = dmin; d <= n; ++d) {
        if (n % d) continue;
        uint32_t qq = (uint32_t)(n / d);
        double l2 = orc_log2_eps_block(n, k, qq);
        if (l2 <= le && (m == 0 || m <= qq)) {
            *n_p = (uint32_t)d;
            *q = qq;
            *m_out = m ? m : qq;
            *log2_eps = l2;
            return 0;
        }
    }
    return -3;
}

/*
 * Algorithm 1's own parameter line: n = ceil(24/(2 delta - 1)),
 * q = b * ceil(log2(N / (eps n)) / b), for N samples of b bits.
 * Returns 0, or -2 if delta <= 1/2, -1 on bad arguments.
 */
int orc_alg1_params(double N, uint32_t b, double delta, double eps, uint32_t *n_p, uint32_t *q)
{
    if (!(N > 0) || b == 0 || !(eps > 0) || !(eps < 1)) return -1;
    if (!(delta > 0.5)) return -2;
    double nn = ceil(24.0 / (2.0 * delta - 1.0));
    double qq = (double)b * ceil(log2(N / (eps * nn)) / (double)b);
    *n_p = (uint32_t)nn;
    *q = (uint32_t)qq;
    return 0;
}

/*
 * Ingest: pack nsamples samples of b bits (b <= 16, taken from the low bits of
 * each uint16) into a stream, sample s at stream bits [s*b, (s+1)*b), LSB
 * first (the raw data X = X_1 ... X_N in ({0,1}^b)^N of Sec. 3).
 * out must hold ceil(nsamples*b/32) words and is fully overwritten.
 */
void orc_pack_samples(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint32_t *out)
{
    uint64_t nbits = nsamples * b;
    memset(out, 0, sizeof(uint32_t) * ((nbits + 31) / 32));
    for (uint64_t s = 0; s < nsamples; ++s)
        for (uint32_t j = 0; j < b; ++j)
            if ((samples[s] >> j) & 1u) {
                uint64_t t = s * b + j;
                out[t >> 5] |= (uint32_t)1 << (t & 31);
            }
}

/*
 * Min-entropy monitoring of the raw samples (Sec. 2: the sources' min-entropy
 * H_min(X) = -log2 max_x P(X = x) is the quantity the extractor's parameters
 * rest on).  counts[v] += the number of samples s with (samples[s] & (2^b - 1))
 * == v, for v < 2^b (bits above b ignored, as for the ingest).
 */
void orc_sample_histogram(uint32_t b, const uint16_t *samples, uint64_t nsamples, uint64_t *counts)
{
    uint32_t mask = (uint32_t)((1u << b) - 1u);
    for (uint64_t s = 0; s < nsamples; ++s) counts[samples[s] & mask] += 1;
}

/* The plug-in estimate -log2(max_v counts[v] / sum_v counts[v]); -1 if empty. */
double orc_min_entropy_estimate(uint32_t b, const uint64_t *counts)
{
    uint64_t total = 0, top = 0;
    for (uint64_t v = 0; v < ((uint64_t)1 << b); ++v) {
        total += counts[v];
        if (counts[v] > top) top = counts[v];
    }
    if (!total) return -1.0;
    return -log2((double)top / (double)total);
}

int orc_max_q(void) { return ORC_MAXQ; }

int orc_has_openmp(void)
{
#ifdef _OPENMP
    return omp_get_max_threads();
#else
    return 0;
#endif
}
