"""GPU tests of Algorithm 2 (qext_alg2_*): every output bit against the
oracle's Algorithm 2 for several rates, sample widths, q_1 and Delta
(including Delta = 0, which is Algorithm 1), 2-byte-aligned pointers, and the
plan's bookkeeping (windows, offsets, polynomials, Theorem 3.3's bound)."""
import math

import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.conftest import read_golden
from tests.gpu_util import host_words

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


def units(words: np.ndarray, off: int = 0) -> torch.Tensor:
    """uint32 words as a device uint16 array, placed at a unit offset."""
    u = np.ascontiguousarray(words, dtype=np.uint32).view(np.uint16)
    buf = torch.zeros(u.size + off + 1, dtype=torch.int16, device="cuda")
    buf[off:off + u.size] = torch.from_numpy(u.view(np.int16)).cuda()
    return buf[off:]


@pytest.mark.parametrize("delta,b,q1,Delta,nb,off", [
    (0.99, 16, 16, 1, 6, 0),      # n_p = 25, q = 16 .. 96
    (10.74 / 16, 16, 16, 1, 8, 1),  # the paper's rate: n_p = 71, q = 16 .. 128
    (0.8, 8, 32, 2, 5, 0),        # n_p = 40, q = 32 .. 96
    (0.9, 16, 64, 0, 4, 3),       # Delta = 0: Algorithm 1 at q = 64
    (0.75, 16, 48, 2, 3, 0),      # n_p = 48, q = 48, 80, 112
])
def test_alg2_matches_oracle(delta, b, q1, Delta, nb, off):
    p = qext.qext_alg2_plan_create(delta, b, q1, Delta, nb)
    info = p.info
    n_p = info["n_p"]
    assert n_p == math.ceil(24 / (2 * delta - 1))
    dq = Delta * b
    end = p.block(nb)
    total_in = n_p * sum(q1 + l * dq for l in range(nb))
    assert end["in_bit"] == total_in and end["out_bit"] == sum(q1 + l * dq for l in range(nb))
    words = (total_in + 31) // 32
    x = workloads.random_words(int(q1 + 7 * nb + off), words)
    y = workloads.random_words(int(q1 + 7 * nb + off + 1), words)
    nout = end["out_bit"] // 16
    out = torch.full((nout + 2,), -1, dtype=torch.int16, device="cuda")
    qext.qext_alg2_extract(p, units(x, off), units(y, off), nb, out)
    torch.cuda.synchronize()
    got = out.cpu().numpy().view(np.uint16)
    assert (got[nout:] == 0xFFFF).all(), "wrote past the output"
    want = oracle.extract_alg2(n_p, q1, dq, nb, x, y).view(np.uint16)[:nout]
    assert (got[:nout] == want).all()
    for l in range(nb):
        bl = p.block(l)
        assert bl["q"] == q1 + l * dq and bl["taps"] == oracle.select_poly(bl["q"])[1]
    assert abs(info["log2_error_bound"] - oracle.alg2_log2_error(n_p, delta, q1, dq, nb)) < 1e-9


def test_alg2_q_up_to_256_oracle_search():
    """q = 16 .. 256 in steps of 48, the oracle searching every field itself."""
    p = qext.qext_alg2_plan_create(0.99, 16, 16, 3, 6)
    n_p = p.info["n_p"]
    total_in = n_p * sum(16 + 48 * l for l in range(6))
    x = workloads.random_words(77, (total_in + 31) // 32)
    y = workloads.random_words(78, (total_in + 31) // 32)
    nout = sum(16 + 48 * l for l in range(6)) // 16
    out = torch.empty(nout, dtype=torch.int16, device="cuda")
    qext.qext_alg2_extract(p, units(x), units(y), 6, out)
    torch.cuda.synchronize()
    want = oracle.extract_alg2(n_p, 16, 48, 6, x, y).view(np.uint16)[:nout]
    assert (out.cpu().numpy().view(np.uint16) == want).all()


def test_alg2_128_blocks_up_to_q_2048():
    """A stream of real length: the paper's rate (delta = 10.74/16, so n = 71),
    b = 16, q_1 = 16, Delta = 1: 128 blocks, q_l = 16 .. 2048 (2 x 9,378,816
    input bits), every output bit against the oracle's Algorithm 2 with the
    oracle-written field polynomials (tests/golden/alg2_field_polys.txt), run
    twice on the same plan (the device sums are cleared per call)."""
    golden = {int(q): tuple(int(t) for t in (c, b, a) if int(t))
              for q, c, b, a in read_golden("alg2_field_polys.txt")}
    p = qext.qext_alg2_plan_create(10.74 / 16, 16, 16, 1, 128)
    n_p = p.info["n_p"]
    assert n_p == 71
    end = p.block(128)
    assert end["in_bit"] == 71 * 16 * 128 * 129 // 2 and end["out_bit"] == 16 * 128 * 129 // 2
    words = (end["in_bit"] + 31) // 32
    x = workloads.random_words(91, words)
    y = workloads.random_words(92, words)
    nout = end["out_bit"] // 16
    taps = [golden[16 * (l + 1)] for l in range(128)]
    want = oracle.extract_alg2(n_p, 16, 16, 128, x, y, taps=taps).view(np.uint16)[:nout]
    for _ in range(2):
        out = torch.full((nout + 2,), -1, dtype=torch.int16, device="cuda")
        qext.qext_alg2_extract(p, units(x), units(y), 128, out)
        torch.cuda.synchronize()
        got = out.cpu().numpy().view(np.uint16)
        assert (got[nout:] == 0xFFFF).all(), "wrote past the output"
        bad = np.nonzero(got[:nout] != want)[0]
        assert bad.size == 0, "first mismatching output unit %d" % bad[0]
    # a prefix of the plan's blocks: the first 40 outputs are the same
    out = torch.full((nout + 2,), -1, dtype=torch.int16, device="cuda")
    qext.qext_alg2_extract(p, units(x), units(y), 40, out)
    torch.cuda.synchronize()
    n40 = p.block(40)["out_bit"] // 16
    assert (out.cpu().numpy().view(np.uint16)[:n40] == want[:n40]).all()
