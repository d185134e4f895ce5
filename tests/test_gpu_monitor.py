"""GPU tests of the min-entropy monitor: the device histogram equals the
oracle's for every sample width class (shared-memory bins up to 13 bits,
global counts above), with junk above b, unaligned starts and ragged tails,
accumulates over chunks, and gives the oracle's estimate."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


@pytest.mark.parametrize("b,n,off", [(8, 1 << 20, 0), (12, (1 << 21) + 5, 0), (12, 1001, 3), (13, 77777, 1),
                                     (14, 300001, 0), (16, 123457, 2), (1, 999, 0), (4, 64, 0)])
def test_histogram_matches_oracle(b, n, off):
    rng = np.random.Generator(np.random.PCG64(b * 1000 + off))
    s = workloads.adc_samples(b + off, n, b) | (rng.integers(0, 1 << 16, n).astype(np.uint16) & np.uint16(0xFFFF ^ ((1 << b) - 1)))
    buf = torch.zeros(n + off, dtype=torch.int16, device="cuda")
    buf[off:] = torch.from_numpy(s.view(np.int16)).cuda()
    counts = torch.zeros(1 << b, dtype=torch.int64, device="cuda")
    qext.qext_sample_histogram(b, buf[off:], n, counts)
    torch.cuda.synchronize()
    got = counts.cpu().numpy().view(np.uint64)
    want = oracle.sample_histogram(b, s)
    assert (got == want).all()
    assert qext.qext_min_entropy_estimate(b, got) == oracle.min_entropy_estimate(b, want)


def test_accumulates_over_chunks_of_a_drifting_stream():
    n = 1 << 22
    s = workloads.adc_samples(9, n, 12, drift_amp=0.05)
    d = torch.from_numpy(s.view(np.int16)).cuda()
    counts = torch.zeros(4096, dtype=torch.int64, device="cuda")
    for c in range(4):
        qext.qext_sample_histogram(12, d[c * n // 4:], n // 4, counts)
    torch.cuda.synchronize()
    assert (counts.cpu().numpy().view(np.uint64) == oracle.sample_histogram(12, s)).all()
