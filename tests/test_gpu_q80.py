"""GPU tests of the q = 80 path (the paper's own field, Sec. 4.2: n_p = 71,
5680-bit blocks of 16-bit samples; any n_p): every output bit against the
oracle, for several n_p, truncations m, ragged block counts, 4-byte-aligned
pointers, and 16-bit raw samples."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.gpu_util import dev_words, host_words, oracle_extract, plan_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


def paper_plan(m: int = 80):
    p = qext.qext_plan_create(5680, m, 0.67125 * 5680, 2.0 ** -30)
    assert (p.info["q"], p.info["n_p"], p.info["gpu_supported"]) == (80, 71, 2)
    return p


def run(plan, nblocks, seed, off=0):
    info = plan.info
    n = info["q"] * info["n_p"]
    words = -(-nblocks * n // 32)
    x = workloads.random_words(seed, words)
    y = workloads.random_words(seed + 1, words)
    nout = -(-nblocks * info["m"] // 32)
    out = torch.full((nout + 3,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract(plan, dev_words(x, offset_words=off), dev_words(y, offset_words=off), nblocks, out)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[nout:] == 0xFFFFFFFF).all(), "wrote past the output"
    want = oracle_extract(plan, x, y, nblocks)
    assert (got[:nout] == want).all(), (info, nblocks)


@pytest.mark.parametrize("nblocks,off", [(1, 0), (2, 1), (31, 0), (32, 0), (33, 3), (97, 0), (97, 1), (1000, 0)])
def test_paper_parameters_match_oracle(nblocks, off):
    run(paper_plan(), nblocks, 100 + nblocks, off)


@pytest.mark.parametrize("n_p,m", [(25, 0), (32, 0), (33, 64), (40, 71), (64, 33), (71, 16), (96, 7), (71, 79),
                                   (340, 0), (400, 50)])
def test_other_shapes_and_truncations(n_p, m):
    """n_p = 340: the largest tiles of 32 blocks (one CTA per SM); n_p = 400:
    too large for them, one block per thread."""
    run(plan_for(80, n_p, m), 301, 7 * n_p + m)


def test_samples_b16_match_oracle():
    plan = paper_plan()
    nblocks = 777
    ns = nblocks * 5680 // 16 + 5
    sx = workloads.adc_samples(31, ns, 16)
    sy = workloads.adc_samples(32, ns, 16)
    nout = -(-nblocks * 80 // 32)
    out = torch.full((nout + 2,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract_samples(plan, 16, torch.from_numpy(sx.view(np.int16)).cuda(),
                              torch.from_numpy(sy.view(np.int16)).cuda(), ns, nblocks, out)
    torch.cuda.synchronize()
    got = host_words(out)
    words = -(-nblocks * 5680 // 32)
    want = oracle_extract(plan, oracle.pack_samples(16, sx)[:words], oracle.pack_samples(16, sy)[:words], nblocks)
    assert (got[:nout] == want).all() and (got[nout:] == 0xFFFFFFFF).all()
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract_samples(plan, 12, 16, 16, ns, 1, 16)
    assert e.value.code == qext.QEXT_E_UNSUPPORTED


def check_sampled(plan, x, y, got, nblocks, seed):
    """Blocks drawn at random (plus both ends), each recomputed by the oracle
    alone from its own 5680 bits, re-based on a word boundary."""
    rng = np.random.Generator(np.random.PCG64(seed))
    for l in np.unique(np.concatenate([rng.integers(0, nblocks, 200), [0, 1, nblocks - 2, nblocks - 1]])):
        l = int(l)
        # block l is bits [5680 l, 5680 (l+1))
        bits0 = 5680 * l
        w0, sh = bits0 // 32, bits0 % 32
        def blockwords(a):
            seg = a[w0:w0 + 179].astype(np.uint64)
            seg = np.concatenate([seg, np.zeros(1, np.uint64)])
            return (((seg[:-1] >> np.uint64(sh)) | (seg[1:] << np.uint64(32 - sh))) & np.uint64(0xFFFFFFFF)).astype(
                np.uint32) if sh else a[w0:w0 + 178].astype(np.uint32)
        z = oracle_extract(plan, blockwords(x), blockwords(y), 1)
        want = int(z[0]) | (int(z[1]) << 32) | (int(z[2]) << 64)
        have = 0
        for i in range(3):
            have |= int(got[(80 * l) // 32 + i]) << (32 * i) if (80 * l) // 32 + i < got.size else 0
        have = (have >> ((80 * l) % 32)) & ((1 << 80) - 1)
        assert have == want, l


def test_large_launch_sampled():
    """2^16 blocks (one launch covering every SM several times), sampled
    blocks checked against the oracle one by one."""
    plan = paper_plan()
    nblocks = 1 << 16
    words = nblocks * 5680 // 32
    x = workloads.random_words(5, words)
    y = workloads.random_words(6, words)
    out = torch.empty(nblocks * 80 // 32, dtype=torch.int32, device="cuda")
    qext.qext_extract(plan, dev_words(x), dev_words(y), nblocks, out)
    torch.cuda.synchronize()
    check_sampled(plan, x, y, host_words(out), nblocks, 3)


def test_paper_workload_full_size_sampled():
    """The paper's parameters at the size and in the launch the benchmark
    times: 2^18 block pairs of seeded 16-bit ADC samples (seeds 51 / 52)
    through qext_extract_samples; the packed stream of 16-bit samples is the
    samples' little-endian words."""
    plan = qext.qext_plan_create(5680, 80, 0.67125 * 5680, 2.0 ** -30)
    assert (plan.info["q"], plan.info["n_p"], plan.info["m"]) == (80, 71, 80)
    nb = 1 << 18
    ns = nb * 5680 // 16
    sx = workloads.adc_samples(51, ns, 16)
    sy = workloads.adc_samples(52, ns, 16)
    out = torch.full((nb * 80 // 32 + 1,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract_samples(plan, 16, torch.from_numpy(sx.view(np.int16)).cuda(),
                              torch.from_numpy(sy.view(np.int16)).cuda(), ns, nb, out)
    torch.cuda.synchronize()
    got = host_words(out)
    assert got[-1] == 0xFFFFFFFF, "wrote past the output"
    check_sampled(plan, oracle.pack_samples(16, sx), oracle.pack_samples(16, sy), got[:-1], nb, 5)


def test_bounded_wait_times_out_and_context_survives():
    """Failure detection in the blocks-in-lanes kernel without a fault: with
    QEXT_F_TEST_TIMEOUT every CTA arms its tile barrier but issues no bulk
    copy, so its bounded wait runs out; the kernel records QEXT_E_TIMEOUT and
    returns, the host reads (and clears) the status, and the next launch on
    the same context is bit-exact.  The mode needs bulk-copied tiles only."""
    plan = paper_plan()
    nblocks = 32 * 40
    words = nblocks * 5680 // 32
    x = workloads.random_words(71, words)
    y = workloads.random_words(72, words)
    tx, ty = dev_words(x), dev_words(y)
    out = torch.full((nblocks * 80 // 32,), -1, dtype=torch.int32, device="cuda")
    assert qext.qext_device_status() == qext.QEXT_OK
    qext.qext_extract_ex(plan, tx, ty, nblocks, out, None, qext.QEXT_F_TEST_TIMEOUT)
    torch.cuda.synchronize()
    assert qext.qext_device_status() == qext.QEXT_E_TIMEOUT
    assert qext.qext_device_status() == qext.QEXT_OK          # read clears it
    qext.qext_extract(plan, tx, ty, nblocks, out)
    torch.cuda.synchronize()
    assert (host_words(out) == oracle_extract(plan, x, y, nblocks)).all()
    assert qext.qext_device_status() == qext.QEXT_OK
    for args, flags in [((tx, ty, nblocks - 1), qext.QEXT_F_TEST_TIMEOUT),        # a ragged last tile
                        ((dev_words(x, offset_words=1), dev_words(y, offset_words=1), nblocks),
                         qext.QEXT_F_TEST_TIMEOUT),                              # no bulk copies
                        ((tx, ty, nblocks), qext.QEXT_F_DIRECT)]:               # no launch options
        with pytest.raises(qext.QextError) as e:
            qext.qext_extract_ex(plan, *args, out, None, flags)
        assert e.value.code == qext.QEXT_E_INVAL
