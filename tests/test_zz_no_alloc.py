"""qext_batch_run_noalloc: the allocation-free batch entry point, for callers
that cannot allocate device memory (a fixed device-memory budget set at
start-up, or a latency-critical loop where cudaMalloc would synchronise the
device).  It must give exactly the outputs of the allocating entry point
(qext_batch_create + qext_batch_run) and of the CPU oracle, call after call,
although every call reuses the same static device scratch; and it must refuse
a stream under CUDA-graph capture, whose recorded descriptor copy would read
a host buffer that the next call rewrites.  This file is collected last."""
import numpy as np
import pytest
import torch

from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.gpu_util import dev_words, host_words, oracle_extract, plan_for

pytestmark = pytest.mark.gpu

SPECS = [  # q, n_p, m, nblocks, pointer offset in words
    (16, 64, 16, 3000, 0), (4, 64, 4, 5000, 0), (64, 64, 64, 400, 0), (8, 64, 5, 129, 1), (1, 64, 1, 300, 0),
    (32, 64, 32, 65, 2), (16, 64, 13, 257, 1), (64, 71, 41, 70, 0), (4, 72, 4, 600, 1), (16, 64, 16, 0, 0),
]


def make(specs, seed):
    rng = np.random.Generator(np.random.PCG64(seed))
    ref_items, na_items, host = [], [], []
    for q, n_p, m, nb, off in specs:
        plan = plan_for(q, n_p, m)
        words = nb * q * n_p // 32
        hx = workloads.random_words(int(rng.integers(1 << 30)), words)
        hy = workloads.random_words(int(rng.integers(1 << 30)), words)
        x = dev_words(hx, offset_words=off)
        y = dev_words(hy, offset_words=off)
        nout = -(-nb * plan.info["m"] // 32)
        ref = torch.full((nout + 2,), -1, dtype=torch.int32, device="cuda")
        na = torch.full((nout + 2,), -1, dtype=torch.int32, device="cuda")
        ref_items.append((plan, x, y, nb, ref))
        na_items.append((plan, x, y, nb, na))
        host.append((hx, hy))
    return ref_items, na_items, host


def test_noalloc_matches_allocating_entry_point_twice():
    qbuild.build()
    # two calls in a row, with different streams and data, on one CUDA stream
    for call, (specs, seed) in enumerate([(SPECS, 1), (SPECS[::-1][:7], 2)]):
        ref_items, na_items, host = make(specs, seed)
        b = qext.qext_batch_create(ref_items)
        qext.qext_batch_run(b)
        qext.qext_batch_run_noalloc(na_items)
        torch.cuda.synchronize()
        for (plan, _, _, nb, ref), (_, _, _, _, na), (hx, hy) in zip(ref_items, na_items, host):
            r, a = host_words(ref), host_words(na)
            assert (r == a).all(), (call, plan.info)          # bit-exact, the tests' tolerance
            assert (a[-2:] == 0xFFFFFFFF).all()
            assert (a[:-2] == oracle_extract(plan, hx, hy, nb)).all(), (call, plan.info)
        b.close()
    assert qext.qext_device_status() == qext.QEXT_OK


def test_noalloc_rejects_too_many_items():
    qbuild.build()
    plan = plan_for(16, 64)
    items = [(plan, 16, 16, 0, 16)] * (qext.QEXT_NOALLOC_MAX_ITEMS + 1)
    with pytest.raises(qext.QextError) as e:
        qext.qext_batch_run_noalloc(items)
    assert e.value.code == qext.QEXT_E_LIMIT


def test_noalloc_refuses_a_capturing_stream():
    qbuild.build()
    _, na_items, _ = make(SPECS[:2], 3)
    qext.qext_batch_run_noalloc(na_items)   # the device's one-time set-up, outside any capture
    torch.cuda.synchronize()
    side = torch.cuda.Stream()
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=side):
        with pytest.raises(qext.QextError) as e:
            qext.qext_batch_run_noalloc(na_items, side)
    assert e.value.code == qext.QEXT_E_STATE
    qext.qext_batch_run_noalloc(na_items)   # still usable afterwards
    torch.cuda.synchronize()
    assert qext.qext_device_status() == qext.QEXT_OK
