"""Serving scheduler on the CPU (fake executor: the same admission, ordering
and batching logic, no GPU): per-channel order, chaining of partial blocks
across requests, the HBM budget, and request validation."""
import numpy as np
import pytest

from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()


def plan(n, k, eps):
    return qext.qext_plan_create(n, 0, k, eps)


def test_order_chaining_and_budget():
    p16 = plan(1024, 867, 2.0 ** -50)
    p4 = plan(256, 202, 2.0 ** -9)
    s = qext.qext_server_create(hbm_budget_bytes=1 << 20, max_batch=8, fake_executor=True)
    chans = [qext.qext_server_add_channel(s, p16 if c % 2 else p4) for c in range(5)]
    rng = np.random.Generator(np.random.PCG64(1))
    expect = {c: [] for c in chans}
    tails = {c: 0 for c in chans}
    rid_chan = {}
    for i in range(200):
        c = int(rng.choice(chans))
        n = 1024 if c % 2 else 256
        bits = int(rng.integers(1, 20 * n))
        rid = qext.qext_server_submit(s, c, 0, 0, 0, bits, 0, bits // n * 16 + 64)
        v = tails[c] + bits
        expect[c].append((rid, v // n))
        tails[c] = v % n
        rid_chan[rid] = c
    qext.qext_server_drain(s, 30.0)
    done = qext.qext_server_poll(s, 1000)
    assert len(done) == 200 and all(d["status"] == qext.QEXT_OK for d in done)
    by_chan = {c: [d for d in done if d["channel"] == c] for c in chans}
    for c in chans:
        got = [(d["request_id"], d["blocks"]) for d in by_chan[c]]
        assert got == expect[c]                           # arrival order kept, tails carried
        m = 16 if c % 2 else 4
        assert all(d["out_bits"] == d["blocks"] * m for d in by_chan[c])
    st = qext.qext_server_get_stats(s)
    assert st["completed"] == st["submitted"] == 200
    assert st["peak_bytes"] <= st["budget_bytes"] == 1 << 20
    assert st["bytes_in_use"] == 0
    s.close()


def test_budget_limits_concurrency():
    p = plan(1024, 867, 2.0 ** -50)
    bits = 64 * 1024
    s = qext.qext_server_create(hbm_budget_bytes=64 * 1024, max_batch=64, fake_executor=True)
    chans = [qext.qext_server_add_channel(s, p) for _ in range(16)]
    for c in chans:
        qext.qext_server_submit(s, c, 0, 0, 0, bits, 0, 1024)
    qext.qext_server_drain(s, 30.0)
    st = qext.qext_server_get_stats(s)
    assert st["completed"] == 16 and st["peak_bytes"] <= 64 * 1024
    assert st["rounds"] >= 4                              # 16 requests of ~17 KB cannot share one round
    s.close()


def test_submit_validation():
    p = plan(1024, 867, 2.0 ** -50)
    s = qext.qext_server_create(hbm_budget_bytes=1 << 16, max_batch=4, fake_executor=True)
    c = qext.qext_server_add_channel(s, p)
    with pytest.raises(qext.QextError) as e:
        qext.qext_server_submit(s, c, 0, 0, 0, 1 << 20, 0, 1 << 20)      # larger than the whole budget
    assert e.value.code == qext.QEXT_E_BUDGET
    with pytest.raises(qext.QextError) as e:
        qext.qext_server_submit(s, c, 0, 0, 0, 4096, 0, 1)               # output buffer too small
    assert e.value.code == qext.QEXT_E_NOSPACE
    with pytest.raises(qext.QextError) as e:
        qext.qext_server_submit(s, 7, 0, 0, 0, 4096, 0, 64)              # no such channel
    assert e.value.code == qext.QEXT_E_INVAL
    with pytest.raises(qext.QextError):
        qext.qext_server_create(hbm_budget_bytes=1 << 20, max_batch=0, fake_executor=True)
    s.close()
