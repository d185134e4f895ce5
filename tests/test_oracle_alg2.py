"""Pins of the oracle's Algorithm 2 (Ext_bs^neq, Sec. 3.3; Theorem 3.3):
the paper's own reduction to Algorithm 1 at Delta = 0, the closed-form
cursor and output offsets (each block equals Ext_IP^{n,q_l} on its window,
recomputed here from closed forms), the output length m_k, bilinearity and
symmetry, and Theorem 3.3's chain of bounds."""
import math

import numpy as np
import pytest

import oracle
from paper_2402_14607_gb300 import workloads


@pytest.fixture(scope="module", autouse=True)
def built():
    oracle.build()


def bits_of(words: np.ndarray) -> int:
    return int.from_bytes(np.ascontiguousarray(words, dtype="<u4").tobytes(), "little")


@pytest.mark.parametrize("q,n_p", [(16, 25), (24, 71), (32, 30)])
def test_delta_zero_is_algorithm1(q, n_p):
    """Sec. 3.3: with Delta = 0 Algorithm 2 becomes Algorithm 1."""
    nb = 5
    x = workloads.random_words(q, (nb * q * n_p + 31) // 32)
    y = workloads.random_words(q + 1, (nb * q * n_p + 31) // 32)
    want = oracle.extract(q, n_p, q, oracle.select_poly(q)[0], x, y, nb)
    assert (oracle.extract_alg2(n_p, q, 0, nb, x, y) == want).all()


@pytest.mark.parametrize("n_p,q1,dq,nb", [(25, 16, 16, 5), (27, 8, 8, 6), (30, 12, 12, 4), (71, 16, 16, 3)])
def test_blocks_are_ext_ip_on_closed_form_windows(n_p, q1, dq, nb):
    """Block l (0-based) has q_l = q1 + l*dq, its window starts at stream bit
    n_p * (l*q1 + dq*l*(l-1)/2) and its output at bit l*q1 + dq*l*(l-1)/2
    (closed forms of the cursor and of Theorem 3.3's m_k)."""
    total_q = nb * q1 + dq * nb * (nb - 1) // 2
    words = (n_p * total_q + 31) // 32
    x = workloads.random_words(3 * n_p + q1, words)
    y = workloads.random_words(3 * n_p + q1 + 1, words)
    out = bits_of(oracle.extract_alg2(n_p, q1, dq, nb, x, y))
    assert out >> total_q == 0, "bits past m_k"
    X, Y = bits_of(x), bits_of(y)
    for l in range(nb):
        ql = q1 + l * dq
        start = n_p * (l * q1 + dq * l * (l - 1) // 2)
        xs = [(X >> (start + e * ql)) & ((1 << ql) - 1) for e in range(n_p)]
        ys = [(Y >> (start + e * ql)) & ((1 << ql) - 1) for e in range(n_p)]
        want = oracle.ext_ip(ql, oracle.select_poly(ql)[0], xs, ys)
        o = l * q1 + dq * l * (l - 1) // 2
        assert (out >> o) & ((1 << ql) - 1) == want, l


def test_bilinear_symmetric_zero():
    n_p, q1, dq, nb = 25, 16, 16, 4
    words = (n_p * (nb * q1 + dq * nb * (nb - 1) // 2) + 31) // 32
    x = workloads.random_words(41, words)
    x2 = workloads.random_words(42, words)
    y = workloads.random_words(43, words)
    a = oracle.extract_alg2(n_p, q1, dq, nb, x, y)
    assert (a == oracle.extract_alg2(n_p, q1, dq, nb, y, x)).all()
    assert (a ^ oracle.extract_alg2(n_p, q1, dq, nb, x2, y) == oracle.extract_alg2(n_p, q1, dq, nb, x ^ x2, y)).all()
    assert not oracle.extract_alg2(n_p, q1, dq, nb, np.zeros_like(x), y).any()


@pytest.mark.parametrize("delta,b,q1,Delta", [(10.74 / 16, 16, 16, 1), (0.8, 8, 16, 2), (0.86, 12, 24, 1)])
def test_theorem33_bound_chain(delta, b, q1, Delta):
    """With n = ceil(24/(2 delta - 1)): sqrt(3) sum 2^(-1/4-(delta/4-1/8) q_l n + 2 q_l)
    <= sqrt(3) sum 2^(-1/4 - q_l) < sqrt(3) 2^(-1/4-q1) / (1 - 2^(-Delta b))."""
    n_p = math.ceil(24 / (2 * delta - 1))
    dq = Delta * b
    for k in (1, 5, 40):
        got = oracle.alg2_log2_error(n_p, delta, q1, dq, k)
        mid = 0.5 * math.log2(3) + math.log2(sum(2.0 ** (-0.25 - (q1 + l * dq)) for l in range(k)))
        top = 0.5 * math.log2(3) - 0.25 - q1 - math.log2(1 - 2.0 ** (-dq))
        # the last step is strict in exact arithmetic (a partial geometric sum);
        # in doubles the tail 2^(-dq k) can fall below the precision
        assert got <= mid + 1e-9 and mid <= top + 1e-12
        # the sum of Theorem 3.1's per-block bounds (Theorem 3.3's first line)
        per = sum(2.0 ** oracle.log2_eps_block(n_p * (q1 + l * dq), delta * n_p * (q1 + l * dq), q1 + l * dq)
                  for l in range(k))
        assert abs(got - math.log2(per)) < 1e-9


def test_rejects_fields_past_the_largest():
    assert oracle.max_q() == 2048
    x = np.zeros(1 << 22, np.uint32)
    with pytest.raises(ValueError):
        oracle.extract_alg2(25, 2048, 16, 2, x, x)   # q_2 = 2064 > 2048
