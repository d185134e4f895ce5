"""GPU tests of the batched persistent launch (qext_batch_*): every stream of a
mixed batch (uneven lengths, q in {1..64}, truncated outputs, 4-byte-aligned
buffers) matches the oracle bit for bit, through plain runs, CUDA-graph
replays with refilled inputs, and every autotuner configuration."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.gpu_util import bits_at, dev_words, host_words, oracle_extract, plan_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


def make_items(specs, seed):
    """specs: (q, n_p, m, nblocks, pointer offset words).  Returns batch items
    plus the host inputs for the oracle."""
    rng = np.random.Generator(np.random.PCG64(seed))
    items, hosts = [], []
    for i, (q, n_p, m, nb, off) in enumerate(specs):
        plan = plan_for(q, n_p, m)
        words = nb * q * n_p // 32
        x = workloads.random_words(int(rng.integers(1 << 30)), words)
        y = workloads.random_words(int(rng.integers(1 << 30)), words)
        nout = -(-nb * plan.info["m"] // 32)
        out = torch.full((nout + 4,), -1, dtype=torch.int32, device="cuda")
        items.append((plan, dev_words(x, offset_words=off), dev_words(y, offset_words=off), nb, out))
        hosts.append((plan, x, y, nb, nout))
    return items, hosts


def expected(hosts):
    return [oracle_extract(plan, x, y, nb) if nb else np.zeros(0, np.uint32) for plan, x, y, nb, _ in hosts]


def check(items, hosts, wants=None):
    torch.cuda.synchronize()
    wants = wants if wants is not None else expected(hosts)
    for (plan, _, _, _, out), (_, x, y, nb, nout), want in zip(items, hosts, wants):
        got = host_words(out)
        assert (got[nout:] == 0xFFFFFFFF).all(), "wrote past the output"
        assert (got[:nout] == want).all(), plan.info


MIXED = [
    (16, 64, 16, 1000, 0), (4, 64, 4, 3000, 0), (64, 64, 64, 300, 0), (8, 64, 8, 129, 0), (1, 64, 1, 700, 1),
    (32, 64, 32, 65, 0), (2, 64, 2, 33, 3), (16, 64, 13, 257, 1), (64, 71, 41, 70, 2), (4, 64, 3, 31, 0),
    (16, 70, 16, 45, 1), (64, 64, 64, 1, 0), (16, 64, 16, 0, 0), (4, 72, 4, 600, 1),
    (64, 40, 64, 100, 0), (64, 72, 50, 70, 1),   # q = 64 with a partial last group
]


def test_mixed_batch_matches_oracle():
    items, hosts = make_items(MIXED, 1)
    b = qext.qext_batch_create(items)
    qext.qext_batch_run(b)
    check(items, hosts)
    b.close()


def test_graph_replay_with_refilled_inputs():
    items, hosts = make_items(MIXED[:6], 2)
    b = qext.qext_batch_create(items)
    s = torch.cuda.Stream()
    qext.qext_batch_capture(b, s)
    qext.qext_batch_launch(b, s)
    s.synchronize()
    check(items, hosts)
    # refill the same buffers with new data, replay the graph
    rng = np.random.Generator(np.random.PCG64(3))
    new_hosts = []
    for (plan, tx, ty, nb, out), (_, _, _, _, nout) in zip(items, hosts):
        words = nb * plan.info["n"] // 32
        x = workloads.random_words(int(rng.integers(1 << 30)), words)
        y = workloads.random_words(int(rng.integers(1 << 30)), words)
        if words:
            tx[:words] = torch.from_numpy(x.view(np.int32)).cuda()
            ty[:words] = torch.from_numpy(y.view(np.int32)).cuda()
        new_hosts.append((plan, x, y, nb, nout))
    torch.cuda.synchronize()
    qext.qext_batch_launch(b, s)
    s.synchronize()
    check(items, new_hosts)
    b.close()


def test_every_config_and_autotune():
    items, hosts = make_items(MIXED, 4)
    wants = expected(hosts)
    b = qext.qext_batch_create(items)
    for small in (1, 2, 4):
        for mid in (1, 2, 4):
            for ctas in (1, 2, 3):
                for order in (0, 1):
                    qext.qext_batch_set_config(b, small, mid, ctas, order)
                    for _, _, _, _, out in items:
                        out.fill_(-1)
                    qext.qext_batch_run(b)
                    check(items, hosts, wants)
    ms = qext.qext_batch_autotune(b, 2)
    assert ms > 0
    for _, _, _, _, out in items:
        out.fill_(-1)
    qext.qext_batch_run(b)
    check(items, hosts, wants)
    with pytest.raises(qext.QextError):
        qext.qext_batch_set_config(b, 3, 1, 2, 0)
    b.close()


def test_empty_batch_and_launch_before_capture():
    b = qext.qext_batch_create([])
    qext.qext_batch_run(b)
    with pytest.raises(qext.QextError) as e:
        qext.qext_batch_launch(b)
    assert e.value.code == qext.QEXT_E_STATE
    torch.cuda.synchronize()
    b.close()


def test_batched_adc_workload_scaled():
    """The batching workload's shape (64 stream pairs, block counts 2^U,
    n over {256, 1024, 4096}, 8- and 12-bit ADC data) at smaller U, packed by
    qext_pack_samples, one launch; sampled blocks of every stream checked."""
    specs = workloads.config_batched(lo=6, hi=11)
    items, hosts = [], []
    for sp in specs:
        plan = qext.qext_plan_create(sp.n, 0, sp.k, sp.eps)
        assert plan.info["q"] == sp.n // 64
        sx, sy = sp.samples("x"), sp.samples("y")
        words = sp.nbits // 32
        px = torch.empty(-(-sx.size * sp.b // 32), dtype=torch.int32, device="cuda")
        py = torch.empty_like(px)
        qext.qext_pack_samples(sp.b, torch.from_numpy(sx.view(np.int16)).cuda(), sx.size, px)
        qext.qext_pack_samples(sp.b, torch.from_numpy(sy.view(np.int16)).cuda(), sy.size, py)
        nout = -(-sp.nblocks * plan.info["m"] // 32)
        out = torch.full((nout + 1,), -1, dtype=torch.int32, device="cuda")
        items.append((plan, px, py, sp.nblocks, out))
        hosts.append((plan, oracle.pack_samples(sp.b, sx)[:words], oracle.pack_samples(sp.b, sy)[:words], sp, nout))
    b = qext.qext_batch_create(items)
    qext.qext_batch_autotune(b, 1)
    for it in items:
        it[4].fill_(-1)
    qext.qext_batch_run(b)
    torch.cuda.synchronize()
    rng = np.random.Generator(np.random.PCG64(11))
    for (plan, _, _, _, out), (_, ox, oy, sp, nout) in zip(items, hosts):
        got = host_words(out)
        assert got[nout] == 0xFFFFFFFF
        info = plan.info
        poly, _ = oracle.select_poly(info["q"])
        wpb = sp.n // 32
        for l in np.unique(np.concatenate([rng.integers(0, sp.nblocks, 8), [0, sp.nblocks - 1]])):
            l = int(l)
            z = oracle.extract(info["q"], info["n_p"], info["m"], poly, ox[l * wpb:(l + 1) * wpb],
                               oy[l * wpb:(l + 1) * wpb], 1)
            zz = int(z[0]) | (int(z[1]) << 32 if z.size > 1 else 0)
            assert bits_at(got, l * info["m"], info["m"]) == zz
    b.close()


@pytest.mark.parametrize("seed", [21, 22])
def test_batched_raw_samples_match_oracle(seed):
    """qext_batch_create_samples: streams of raw 8-, 12- and 16-bit samples
    (garbage above the low b bits of each uint16), q in {1 .. 64}, ragged
    block counts and spare samples, one launch with the ingest inside; every
    output bit against the oracle on the packed streams, and equal to
    qext_extract_samples / the packed-word batch on the same data."""
    rng = np.random.Generator(np.random.PCG64(seed))
    specs = [(16, 64, 16, 1000, 12), (4, 64, 4, 3000, 8), (64, 64, 64, 300, 12), (64, 64, 50, 129, 8),
             (16, 64, 13, 257, 16), (8, 64, 8, 129, 12), (1, 64, 1, 700, 8), (32, 64, 32, 65, 12),
             (64, 64, 64, 1, 16), (16, 64, 16, 0, 12), (4, 72, 4, 600, 12), (64, 40, 64, 100, 12)]
    items, hosts, packed = [], [], []
    for q, n_p, m, nb, b in specs:
        plan = plan_for(q, n_p, m)
        n = q * n_p
        ns = -(-nb * n // b) + int(rng.integers(0, 20))
        raw_x = rng.integers(0, 1 << 16, ns, dtype=np.uint16)
        raw_y = rng.integers(0, 1 << 16, ns, dtype=np.uint16)
        sx = torch.from_numpy(raw_x.view(np.int16)).cuda()
        sy = torch.from_numpy(raw_y.view(np.int16)).cuda()
        nout = -(-nb * plan.info["m"] // 32)
        out = torch.full((nout + 2,), -1, dtype=torch.int32, device="cuda")
        items.append((plan, b, sx, sy, ns, nb, out))
        words = nb * n // 32
        hosts.append((plan, oracle.pack_samples(b, raw_x)[:words], oracle.pack_samples(b, raw_y)[:words], nb, nout))
        px = torch.empty(max(1, -(-ns * b // 32)), dtype=torch.int32, device="cuda")
        py = torch.empty_like(px)
        if ns:
            qext.qext_pack_samples(b, sx, ns, px)
            qext.qext_pack_samples(b, sy, ns, py)
        packed.append((plan, px, py, nb, torch.full((nout + 2,), -1, dtype=torch.int32, device="cuda")))
    bs = qext.qext_batch_create_samples(items)
    qext.qext_batch_run(bs)
    wants = expected(hosts)
    check([(it[0], None, None, it[5], it[6]) for it in items], hosts, wants)
    bp = qext.qext_batch_create(packed)
    qext.qext_batch_run(bp)
    torch.cuda.synchronize()
    for it, pk in zip(items, packed):
        assert torch.equal(it[6], pk[4])
    # graph replay and every configuration give the same bits
    s = torch.cuda.Stream()
    for cfg in [(1, 1, 1, 1), (2, 2, 2, 0), (4, 4, 3, 0)]:
        qext.qext_batch_set_config(bs, *cfg)
        for it in items:
            it[6].fill_(-1)
        qext.qext_batch_capture(bs, s)
        qext.qext_batch_launch(bs, s)
        s.synchronize()
        check([(it[0], None, None, it[5], it[6]) for it in items], hosts, wants)
    # the test mode of failure detection needs bulk-copied tiles
    with pytest.raises(qext.QextError) as e:
        qext.qext_batch_run_ex(bs, None, qext.QEXT_F_TEST_TIMEOUT)
    assert e.value.code == qext.QEXT_E_INVAL
    bs.close()
    bp.close()


def test_batched_bounded_wait_times_out_and_context_survives():
    """Failure detection in the batched kernel without a fault: each CTA arms
    its tile barrier but no bulk copy is issued, so its bounded wait runs out;
    the kernel records QEXT_E_TIMEOUT and returns, the host reads (and clears)
    the status, and the next run on the same context is correct."""
    specs = [(16, 64, 16, 2000, 0), (64, 64, 64, 300, 0), (4, 64, 4, 5000, 0)]
    items, hosts = make_items(specs, 41)
    b = qext.qext_batch_create(items)
    assert qext.qext_device_status() == qext.QEXT_OK
    qext.qext_batch_run_ex(b, None, qext.QEXT_F_TEST_TIMEOUT)
    torch.cuda.synchronize()
    assert qext.qext_device_status() == qext.QEXT_E_TIMEOUT
    assert qext.qext_device_status() == qext.QEXT_OK          # read clears it
    qext.qext_batch_run(b)
    torch.cuda.synchronize()
    for it, want in zip(items, expected(hosts)):
        assert (host_words(it[4])[:want.size] == want).all()
    assert qext.qext_device_status() == qext.QEXT_OK
    # the test mode needs every stream on the bulk-copy path
    mis, _ = make_items([(16, 64, 16, 100, 1)], 42)
    b2 = qext.qext_batch_create(mis)
    with pytest.raises(qext.QextError) as e:
        qext.qext_batch_run_ex(b2, None, qext.QEXT_F_TEST_TIMEOUT)
    assert e.value.code == qext.QEXT_E_INVAL
    b2.close()
    b.close()
