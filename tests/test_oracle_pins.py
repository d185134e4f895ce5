"""Pins for the CPU oracle: facts fixed by the paper and by the mathematics,
checked with code written independently of the oracle (Python big-int
polynomial arithmetic, trial division, Berlekamp's matrix, brute force).

Nothing here touches a GPU.  Each test names the passage it pins.
"""
import math
import random

import numpy as np
import pytest

import oracle
from tests.conftest import read_golden


# --------------------------------------------------------------------------
# Independent GF(2)[x] arithmetic on Python ints (full product, then long
# division -- a different algorithm from the oracle's per-shift reduction).
# --------------------------------------------------------------------------
def clmul(a, b):
    r = 0
    while b:
        if b & 1:
            r ^= a
        a <<= 1
        b >>= 1
    return r


def pdeg(a):
    return a.bit_length() - 1


def polymod(a, m):
    dm = pdeg(m)
    while a and pdeg(a) >= dm:
        a ^= m << (pdeg(a) - dm)
    return a


def mulmod(a, b, m):
    return polymod(clmul(a, b), m)


def pgcd(a, b):
    while b:
        a, b = b, polymod(a, b)
    return a


def irreducible_trial_division(p):
    d = pdeg(p)
    for f in range(2, 1 << (d // 2 + 1)):
        if 1 <= pdeg(f) <= d // 2 and polymod(p, f) == 0:
            return False
    return True


def gf2_rank(rows):
    rows = [r for r in rows if r]
    rank = 0
    while rows:
        piv = max(rows, key=pdeg)
        rows.remove(piv)
        top = pdeg(piv)
        rows = [r ^ piv if pdeg(r) == top else r for r in rows]
        rows = [r for r in rows if r]
        rank += 1
    return rank


def irreducible_berlekamp(f):
    """Squarefree (gcd(f, f') = 1) and rank(Q - I) = deg f - 1, where row i of
    Q is x^(2i) mod f: exactly one irreducible factor."""
    n = pdeg(f)
    deriv = 0
    for i in range(1, n + 1):
        if (f >> i) & 1 and i % 2 == 1:
            deriv |= 1 << (i - 1)
    if deriv == 0 or pgcd(f, deriv) != 1:
        return False
    x2 = polymod(4, f)
    r = 1
    rows = []
    for i in range(n):
        rows.append(r ^ (1 << i))
        r = mulmod(r, x2, f)
    return gf2_rank(rows) == n - 1


def candidates_before(q, poly):
    """All minimum-weight-rule candidates that come before ``poly``."""
    out = []
    for a in range(1, q):
        p = (1 << q) | (1 << a) | 1
        if p == poly:
            return out
        out.append(p)
    for c in range(3, q):
        for b in range(2, c):
            for a in range(1, b):
                p = (1 << q) | (1 << c) | (1 << b) | (1 << a) | 1
                if p == poly:
                    return out
                out.append(p)
    raise AssertionError("poly not in candidate order")


def pack_blocks(values, t):
    """Concatenate t-bit values LSB-first into a uint32 stream."""
    values = np.asarray(values, dtype=np.uint64)
    bits = ((values[:, None] >> np.arange(t, dtype=np.uint64)[None, :]) & 1).astype(np.uint8).ravel()
    pad = (-bits.size) % 32
    bits = np.concatenate([bits, np.zeros(pad + 32, np.uint8)])
    return np.packbits(bits.reshape(-1, 8)[:, ::-1]).view("<u4").astype(np.uint32)


def unpack_values(words, m, count):
    bits = np.unpackbits(np.asarray(words, dtype="<u4").view(np.uint8), bitorder="little")
    bits = bits[: m * count].reshape(count, m).astype(np.uint64)
    return (bits << np.arange(m, dtype=np.uint64)[None, :]).sum(axis=1).astype(np.uint64)


# --------------------------------------------------------------------------
# Field multiplication (Sec. 3.2: F_{2^q} in polynomial basis)
# --------------------------------------------------------------------------
def test_fips197_published_products():
    """FIPS-197 Sec. 4.2 / 4.2.1 products in GF(2^8) mod x^8+x^4+x^3+x+1."""
    for a, b, c in read_golden("fips197_gf256_products.txt"):
        assert oracle.gf_mul(8, 0x11B, int(a, 16), int(b, 16)) == int(c, 16)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 8, 12, 16, 31, 32, 33, 63, 64, 80, 127, 200])
def test_gf_mul_matches_independent_bigint(q):
    poly, _ = oracle.select_poly(q)
    rng = random.Random(q)
    for _ in range(40):
        a = rng.getrandbits(q)
        b = rng.getrandbits(q)
        assert oracle.gf_mul(q, poly, a, b) == mulmod(a, b, poly)


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 6])
def test_field_axioms_exhaustive(q):
    poly, _ = oracle.select_poly(q)
    N = 1 << q
    T = np.array([[oracle.gf_mul(q, poly, a, b) for b in range(N)] for a in range(N)], dtype=np.int64)
    assert (T == T.T).all()                                   # commutative
    assert (T[1] == np.arange(N)).all()                       # 1 is the identity
    assert (T[0] == 0).all()
    for a in range(N):                                        # associative, distributive
        for b in range(N):
            assert (T[T[a, b]] == T[a][T[b]]).all()
            assert (T[a][np.arange(N) ^ b] == (T[a] ^ T[a, b])).all()
    for a in range(1, N):                                     # every a != 0 invertible
        assert (T[a] == 1).sum() == 1
    for a in range(N):                                        # a^(2^q) = a
        x = a
        for _ in range(q):
            x = T[x, x]
        assert x == a


@pytest.mark.parametrize("q", [16, 64, 80])
def test_field_axioms_random(q):
    poly, _ = oracle.select_poly(q)
    rng = random.Random(1000 + q)
    mul = lambda a, b: oracle.gf_mul(q, poly, a, b)
    for _ in range(6):
        a, b, c = (rng.getrandbits(q) for _ in range(3))
        assert mul(a, b) == mul(b, a)
        assert mul(mul(a, b), c) == mul(a, mul(b, c))
        assert mul(a, b ^ c) == mul(a, b) ^ mul(a, c)
        x = a
        for _ in range(q):
            x = mul(x, x)
        assert x == a                                          # Frobenius: a^(2^q) = a
        if a:
            inv, base, e = 1, a, (1 << q) - 2                  # a^(2^q - 2) = a^-1
            while e:
                if e & 1:
                    inv = mul(inv, base)
                base = mul(base, base)
                e >>= 1
            assert mul(a, inv) == 1


# --------------------------------------------------------------------------
# Field polynomial choice (minimum weight, lexicographically first)
# --------------------------------------------------------------------------
def test_rabin_agrees_with_trial_division():
    for d in range(1, 11):
        for low in range(0, 1 << d, 1):
            p = (1 << d) | low
            if not p & 1 and d > 1:
                continue
            assert oracle.is_irreducible(d, p) == irreducible_trial_division(p), hex(p)


@pytest.mark.parametrize("q", list(range(2, 17)))
def test_selected_poly_small_q(q):
    poly, taps = oracle.select_poly(q)
    assert pdeg(poly) == q and poly & 1
    assert irreducible_trial_division(poly)
    for p in candidates_before(q, poly):
        assert not irreducible_trial_division(p), hex(p)
    assert bin(poly).count("1") == len(taps) + 2


@pytest.mark.parametrize("q", [24, 32, 48, 64, 80])
def test_selected_poly_large_q_berlekamp(q):
    poly, taps = oracle.select_poly(q)
    assert pdeg(poly) == q
    assert irreducible_berlekamp(poly)
    for p in candidates_before(q, poly):
        assert not irreducible_berlekamp(p), hex(p)
    if q % 8 == 0:          # Swan: no irreducible trinomial of degree 8k
        assert len(taps) == 3


# --------------------------------------------------------------------------
# Ext_IP (Definition 3.2) through the Algorithm 1 block loop
# --------------------------------------------------------------------------
def test_q1_is_textbook_inner_product():
    """q = 1: F_2, Ext = <x, y> mod 2, the Hadamard extractor (CG88)."""
    rng = np.random.Generator(np.random.PCG64(5))
    for n_p in [1, 7, 32, 64, 100]:
        nb = 37
        xv = rng.integers(0, 2, size=(nb, n_p))
        yv = rng.integers(0, 2, size=(nb, n_p))
        to_int = lambda r: int(sum(int(b) << i for i, b in enumerate(r)))
        x = pack_blocks([to_int(r) for r in xv], n_p) if n_p <= 64 else None
        if x is None:
            bits = xv.ravel()
            ybits = yv.ravel()
            x = np.packbits(np.concatenate([bits, np.zeros((-bits.size) % 32 + 32, int)]).astype(np.uint8)
                            .reshape(-1, 8)[:, ::-1]).view("<u4")
            y = np.packbits(np.concatenate([ybits, np.zeros((-ybits.size) % 32 + 32, int)]).astype(np.uint8)
                            .reshape(-1, 8)[:, ::-1]).view("<u4")
        else:
            y = pack_blocks([to_int(r) for r in yv], n_p)
        poly, _ = oracle.select_poly(1)
        out = oracle.extract(1, n_p, 1, poly, x, y, nb)
        got = unpack_values(out, 1, nb)
        want = (xv & yv).sum(axis=1) % 2
        assert (got == want).all()


@pytest.mark.parametrize("q", [4, 16, 64, 80])
def test_np1_is_field_multiplication(q):
    poly, _ = oracle.select_poly(q)
    rng = random.Random(q * 7)
    xs = [rng.getrandbits(q) for _ in range(50)]
    ys = [rng.getrandbits(q) for _ in range(50)]
    out = oracle.extract(q, 1, q, poly, pack_blocks(xs, q) if q <= 64 else _pack_big(xs, q),
                         pack_blocks(ys, q) if q <= 64 else _pack_big(ys, q), 50)
    for i in range(50):
        assert _get_bits(out, i * q, q) == mulmod(xs[i], ys[i], poly)


def _pack_big(values, t):
    acc = 0
    for i, v in enumerate(values):
        acc |= v << (i * t)
    nw = (len(values) * t + 31) // 32 + 1
    return np.array([(acc >> (32 * w)) & 0xFFFFFFFF for w in range(nw)], dtype=np.uint32)


def _get_bits(words, start, count):
    acc = 0
    for w, v in enumerate(words):
        acc |= int(v) << (32 * w)
    return (acc >> start) & ((1 << count) - 1)


@pytest.mark.parametrize("q,n_p", [(4, 64), (16, 64), (64, 64), (80, 71), (3, 5)])
def test_bilinear_symmetric_zero(q, n_p):
    """Ext is F_2-bilinear and symmetric, Ext(0, y) = 0 (Definition 3.2)."""
    poly, _ = oracle.select_poly(q)
    rng = random.Random(q + n_p)
    xs, x2s, ys = ([[rng.getrandbits(q) for _ in range(n_p)] for _ in range(3)])
    e = lambda a, b: oracle.ext_ip(q, poly, a, b)
    assert e(xs, ys) == e(ys, xs)
    assert e([a ^ b for a, b in zip(xs, x2s)], ys) == e(xs, ys) ^ e(x2s, ys)
    assert e([0] * n_p, ys) == 0
    # and the inner product is a sum of field products
    want = 0
    for a, b in zip(xs, ys):
        want ^= mulmod(a, b, poly)
    assert e(xs, ys) == want


def ext_table(q, n_p):
    """T[x, y] = Ext_IP over all pairs of t = q*n_p bit blocks (oracle)."""
    t = q * n_p
    poly, _ = oracle.select_poly(q)
    N = 1 << t
    xstream = pack_blocks(np.arange(N), t)
    T = np.zeros((N, N), dtype=np.int64)
    for yv in range(N):
        ystream = pack_blocks(np.full(N, yv), t)
        out = oracle.extract(q, n_p, q, poly, xstream, ystream, N)
        T[:, yv] = unpack_values(out, q, N).astype(np.int64)
    return T, poly


@pytest.mark.parametrize("q,n_p", [(1, 8), (2, 4), (3, 3), (4, 2), (2, 5), (5, 2)])
def test_exact_uniformity(q, n_p):
    """x uniform on {0,1}^t and y with a nonzero element: Ext(x, y) is exactly
    uniform on {0,1}^q (x -> Ext(x, y) is a surjective linear map)."""
    T, _ = ext_table(q, n_p)
    t = q * n_p
    for yv in range(1, 1 << t):
        counts = np.bincount(T[:, yv], minlength=1 << q)
        assert (counts == (1 << (t - q))).all()
    assert (T[:, 0] == 0).all()


@pytest.mark.parametrize("q,n_p", [(1, 6), (2, 3), (2, 4), (4, 2), (8, 1)])
def test_hadamard_property_prop_a2(q, n_p):
    """Prop. A.2: for a != 0, f_a(x, y) = [a * Ext(x, y)]_1 is a Hadamard
    function, i.e. the +-1 matrix F_a satisfies F_a F_a^T = 2^t I."""
    T, poly = ext_table(q, n_p)
    t = q * n_p
    for a in range(1, 1 << q):
        amul = np.array([oracle.gf_mul(q, poly, a, z) & 1 for z in range(1 << q)], dtype=np.int64)
        F = 1 - 2 * amul[T]
        G = F @ F.T
        assert (G == (1 << t) * np.eye(1 << t, dtype=np.int64)).all()


@pytest.mark.parametrize("q", [1, 2, 3, 4, 5, 8])
def test_s_to_a_bijection(q):
    """Appendix A: every parity S.Z equals the first bit of a*Z for exactly
    one a, and S -> a is a bijection with 0 -> 0."""
    poly, _ = oracle.select_poly(q)
    N = 1 << q
    first_bit = np.array([[oracle.gf_mul(q, poly, a, z) & 1 for z in range(N)] for a in range(N)])
    parity = np.array([[bin(s & z).count("1") & 1 for z in range(N)] for s in range(N)])
    match = {}
    for s in range(N):
        hits = [a for a in range(N) if (first_bit[a] == parity[s]).all()]
        assert len(hits) == 1
        match[s] = hits[0]
    assert sorted(match.values()) == list(range(N))
    assert match[0] == 0


def _dist(T, xs, ys, q):
    sub = T[np.ix_(xs, ys)].ravel()
    return np.bincount(sub, minlength=1 << q) / sub.size


@pytest.mark.parametrize("q,n_p", [(1, 8), (2, 4), (2, 5), (5, 2), (1, 10)])
def test_distance_from_uniform_vs_bounds(q, n_p):
    """Brute-force statistical distance of Ext(X, Y) over flat sources of
    min-entropy k, against CG88's one-bit bound (Lemma A.5), the XOR lemma
    (Lemma 2.4, classical form) and Theorem 3.1's bound."""
    T, poly = ext_table(q, n_p)
    t = q * n_p
    rng = np.random.Generator(np.random.PCG64(t * 31 + q))
    afirst = np.array([[oracle.gf_mul(q, poly, a, z) & 1 for z in range(1 << q)] for a in range(1 << q)])
    for k in range(t // 2 + 1, t):
        for _ in range(4):
            xs = rng.choice(1 << t, size=1 << k, replace=False)
            ys = rng.choice(1 << t, size=1 << k, replace=False)
            P = _dist(T, xs, ys, q)
            sd = 0.5 * np.abs(P - 2.0 ** -q).sum()
            biases = []
            for a in range(1, 1 << q):
                p1 = P[afirst[a] == 1].sum()
                bias = abs(p1 - 0.5)
                assert bias <= 2.0 ** (-(2 * k - t) / 2) + 1e-12         # Lemma A.5: eps/2
                biases.append(bias)
            assert 2 * sd <= (2 ** q) * sum(2 * b for b in biases) + 1e-12   # Lemma 2.4
            delta = k / t
            thm31 = math.sqrt(3) * 2 ** (-0.25 - (delta / 4 - 0.125) * t + 2 * q)
            assert sd <= thm31


def test_adversarial_subspace_sources():
    """q = 1, t = 8: X in a 4-dim subspace V, Y in V^perp gives Ext = 0
    always (distance 1/2), the worst case at rate exactly 1/2; just above
    rate 1/2 the CG88 bound holds."""
    T, _ = ext_table(1, 8)
    V = [v for v in range(256) if v >> 4 == 0]            # span of e0..e3
    W = [w for w in range(256) if w & 0xF == 0]            # span of e4..e7 = V^perp
    P = _dist(T, np.array(V), np.array(W), 1)
    assert P[0] == 1.0
    assert 0.5 * np.abs(P - 0.5).sum() == 0.5


# --------------------------------------------------------------------------
# Parameters: Algorithm 1's line, Theorem 3.1 / 3.3 / 3.4, Sec. 4.2 example
# --------------------------------------------------------------------------
def _golden_example():
    return {r[0]: r[1] for r in read_golden("paper_sec42_worked_example.txt")}


def test_worked_example_parameters():
    g = _golden_example()
    b = int(g["b"])
    delta = float(g["delta_num"]) / float(g["delta_den"])
    N = 2.0 ** int(g["log2_N"])
    eps = 2.0 ** int(g["log2_eps"])
    n_p, q = oracle.alg1_params(N, b, delta, eps)
    assert (n_p, q) == (int(g["n_p"]), int(g["q"]))
    # the per-block plan reaches the same factorisation for a 71*80-bit block
    n = n_p * q
    p = oracle.plan(n, q, delta * n, eps)
    assert (p["n_p"], p["q"]) == (n_p, q)
    assert p["log2_eps"] < math.log2(eps)


def test_worked_example_arithmetic():
    g = _golden_example()
    n_p, q = int(g["n_p"]), int(g["q"])
    ops = q * (n_p - 1) + int(g["gf80_mult_ops"]) * n_p
    assert ops == int(g["ext_ip_ops"])
    units = (int(g["luts"]) * int(g["ops_per_lut"])) // ops
    assert units == int(g["parallel_units"])
    assert int(g["clock_hz"]) * units * q == int(g["speed_bps"])
    out_bits = 2.0 ** int(g["log2_N"]) * int(g["b"]) / n_p       # Theorem 3.4, m = Nb/n
    assert round(out_bits / 2 ** 50, 2) == float(g["output_pb_approx"])
    delta = float(g["delta_num"]) / float(g["delta_den"])
    assert round((2 * delta - 1) / (48 * delta), 4) == float(g["fraction_approx"])


def test_theorem31_constant_chain():
    """Lemma A.6 with k' = (1/4 + delta/2) qn + 1/2 and eps' = 2^(1/2 - (delta/2 -
    1/4) qn) needs min-entropy k' + log2(1/eps') = delta qn and gives
    sqrt(3 eps'/2) = sqrt(3) 2^(-1/4 - (delta/4 - 1/8) qn) (Lemma 3.2); the
    XOR lemma's 2^q over 2^q - 1 parities gives Theorem 3.1's 2^(2q)."""
    for (q, n_p, k) in [(16, 64, 867), (4, 64, 202), (64, 64, 3485), (80, 71, 3812.7)]:
        t = q * n_p
        delta = k / t
        kp = (0.25 + delta / 2) * t + 0.5
        log2_epsp = 0.5 - (delta / 2 - 0.25) * t
        assert abs(kp - log2_epsp - k) < 1e-9
        # Lemma A.5 at k': eps = 2^(1 - (2k' - t)/2) equals eps'
        assert abs((1 - (2 * kp - t) / 2) - log2_epsp) < 1e-9
        one_bit = 0.5 * math.log2(3 * 2 ** log2_epsp / 2)
        lemma32 = 0.5 * math.log2(3) - 0.25 - (delta / 4 - 0.125) * t
        assert abs(one_bit - lemma32) < 1e-9
        # per-parity trace distance 2*lemma32, times 2^q parities, times 2^q,
        # halved: sqrt(3) 2^(..+2q) (Theorem 3.1 reads the sum as < 2^q terms)
        assert abs(oracle.log2_eps_block(t, k, q) - (lemma32 + 2 * q)) < 1e-9


@pytest.mark.parametrize("n,k,eps,want", [
    (256, 202, 2.0 ** -9, (64, 4)),
    (1024, 867, 2.0 ** -50, (64, 16)),
    (1024, 867, 2.0 ** -60, (128, 8)),
    (4096, 3485, 2.0 ** -52, (64, 64)),
    (4096, 3510, 2.0 ** -52, (64, 64)),
])
def test_plan_table(n, k, eps, want):
    p = oracle.plan(n, 0, k, eps)
    assert (p["n_p"], p["q"]) == want
    assert p["m"] == p["q"]
    assert p["log2_eps"] <= math.log2(eps)
    # the chosen n_p is at least Algorithm 1's ceil(24/(2 delta - 1))
    assert p["n_p"] >= math.ceil(24 / (2 * k / n - 1) - 1e-12)
    # and Theorem 3.3's second inequality: eps_blk <= sqrt(3) 2^(-1/4 - q)
    assert p["log2_eps"] <= 0.5 * math.log2(3) - 0.25 - p["q"] + 1e-9


def test_plan_rejections_and_exact_ceiling():
    with pytest.raises(oracle.PlanError):
        oracle.plan(1024, 0, 512, 0.5)             # delta = 1/2
    with pytest.raises(oracle.PlanError):
        oracle.plan(256, 0, 202, 2.0 ** -40)       # unattainable
    # n_min exactly an integer: n = 96, k = 60 -> 24*96/(120-96) = 96 = n_min
    p = oracle.plan(96 * 4, 0, 240, 0.5)           # n = 384, 24*384/(480-384) = 96
    assert p["n_p"] == 96 and p["q"] == 4
    # n = 2048, k = 1800: n_min = 32; d = 32 (q = 64) gives 2^-65.5, d = 64
    # (q = 32) gives 2^-129.5.  The first d meeting eps wins; m must fit in q.
    p = oracle.plan(2048, 40, 1800, 2.0 ** -60)
    assert (p["n_p"], p["q"], p["m"]) == (32, 64, 40)
    p = oracle.plan(2048, 0, 1800, 2.0 ** -100)
    assert (p["n_p"], p["q"], p["m"]) == (64, 32, 32)
    with pytest.raises(oracle.PlanError):
        oracle.plan(2048, 40, 1800, 2.0 ** -100)  # q = 32 < m and larger q misses eps


def test_output_length_theorem34():
    """m = N b / n_p output bits for N samples of b bits (Theorem 3.4)."""
    q, n_p = 16, 64
    poly, _ = oracle.select_poly(q)
    nb = 100
    rng = np.random.Generator(np.random.PCG64(2))
    x = rng.integers(0, 1 << 32, size=nb * q * n_p // 32, dtype=np.uint64).astype(np.uint32)
    y = rng.integers(0, 1 << 32, size=nb * q * n_p // 32, dtype=np.uint64).astype(np.uint32)
    out = oracle.extract(q, n_p, q, poly, x, y, nb)
    assert out.size * 32 == nb * q == (x.size * 32) // n_p


def test_concatenation_and_truncation():
    """Algorithm 1 outputs Z^(1) Z^(2) ... in order: the stream output is the
    concatenation of per-block outputs, each truncated to its first m bits."""
    q, n_p = 16, 64
    poly, _ = oracle.select_poly(q)
    rng = np.random.Generator(np.random.PCG64(3))
    nb = 9
    x = rng.integers(0, 1 << 32, size=nb * 32, dtype=np.uint64).astype(np.uint32)
    y = rng.integers(0, 1 << 32, size=nb * 32, dtype=np.uint64).astype(np.uint32)
    full = oracle.extract(q, n_p, q, poly, x, y, nb)
    for m in [16, 13, 1]:
        tr = oracle.extract(q, n_p, m, poly, x, y, nb)
        for l in range(nb):
            one = oracle.extract(q, n_p, q, poly, x[32 * l:32 * (l + 1)], y[32 * l:32 * (l + 1)], 1)
            assert _get_bits(full, l * q, q) == int(one[0]) & 0xFFFF
            assert _get_bits(tr, l * m, m) == int(one[0]) & ((1 << m) - 1)
        assert int(tr[-1]) >> ((nb * m) % 32 or 32) == 0 if (nb * m) % 32 else True


def test_openmp_matches_single_thread():
    q, n_p = 16, 64
    poly, _ = oracle.select_poly(q)
    rng = np.random.Generator(np.random.PCG64(4))
    nb = 513
    x = rng.integers(0, 1 << 32, size=nb * 32, dtype=np.uint64).astype(np.uint32)
    y = rng.integers(0, 1 << 32, size=nb * 32, dtype=np.uint64).astype(np.uint32)
    a = oracle.extract(q, n_p, 13, poly, x, y, nb, threads=1)
    b = oracle.extract(q, n_p, 13, poly, x, y, nb, threads=0)
    assert (a == b).all()


@pytest.mark.parametrize("b", [1, 8, 12, 16, 7])
def test_pack_samples_lsb_first(b):
    rng = np.random.Generator(np.random.PCG64(b))
    s = rng.integers(0, 1 << b, size=301).astype(np.uint16)
    words = oracle.pack_samples(b, s)
    acc = 0
    for w, v in enumerate(words):
        acc |= int(v) << (32 * w)
    for i, v in enumerate(s):
        assert (acc >> (i * b)) & ((1 << b) - 1) == int(v)
    assert acc >> (301 * b) == 0
