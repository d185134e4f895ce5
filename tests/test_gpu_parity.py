"""GPU parity: libqext's kernels against the CPU oracle, bit for bit, through
the C ABI.  Sizes span several CTAs and warps with ragged tails; block
layouts cover partial element groups and 4-byte-aligned pointers."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.gpu_util import bits_at, dev_words, gpu_extract, host_words, oracle_extract, plan_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


CASES = [
    # q, n_p, m, nblocks, pointer offset in words
    (1, 64, 1, 1000, 0), (1, 96, 1, 77, 1),
    (2, 64, 2, 1000, 0), (2, 48, 1, 333, 1),
    (4, 64, 4, 4099, 0), (4, 64, 3, 1001, 0), (4, 72, 4, 257, 1), (4, 40, 2, 65, 0),
    (8, 64, 8, 1000, 0), (8, 68, 5, 130, 0), (8, 32, 8, 95, 3),
    (16, 64, 16, 4133, 0), (16, 64, 13, 1000, 0), (16, 70, 16, 97, 1), (16, 26, 9, 200, 0), (16, 64, 1, 31, 2),
    (32, 64, 32, 500, 0), (32, 33, 17, 65, 1), (32, 25, 32, 40, 0),
    (64, 64, 64, 300, 0), (64, 71, 41, 70, 1), (64, 64, 1, 100, 0), (64, 25, 64, 33, 0), (64, 64, 63, 257, 2),
    (64, 40, 64, 300, 0), (64, 72, 37, 129, 0), (64, 34, 64, 65, 1),     # q = 64, last group partial
    (64, 64, 64, 1000, 0), (16, 64, 16, 20000, 0), (4, 64, 4, 30001, 0),    # many tiles per CTA
    (16, 800, 16, 70, 0), (64, 200, 64, 40, 0), (8, 1600, 8, 33, 0),        # long blocks: direct fallback
]


@pytest.mark.parametrize("flags", [0, qext.QEXT_F_DIRECT, qext.QEXT_F_CTA_TILES], ids=["default", "direct", "cta_tiles"])
@pytest.mark.parametrize("q,n_p,m,nblocks,off", CASES)
def test_extract_matches_oracle(q, n_p, m, nblocks, off, flags):
    plan = plan_for(q, n_p, m)
    n = q * n_p
    rng = np.random.Generator(np.random.PCG64(q * 1000 + n_p + m))
    words = nblocks * n // 32
    x = workloads.random_words(int(rng.integers(1 << 30)), words)
    y = workloads.random_words(int(rng.integers(1 << 30)), words)
    got = gpu_extract(plan, x, y, nblocks, offset_words=off, flags=flags)
    want = oracle_extract(plan, x, y, nblocks)
    assert got.shape == want.shape
    bad = np.nonzero(got != want)[0]
    assert bad.size == 0, "first mismatching output word %d" % bad[0]


@pytest.mark.parametrize("q", [4, 16, 64])
def test_degenerate_inputs(q):
    """All-zero sources give Z = 0; a zero block on one side zeroes its Z;
    one block and nblocks = 0 work."""
    plan = plan_for(q, 64)
    words = 64 * q // 32
    nb = 70
    x = workloads.random_words(7, nb * words)
    y = workloads.random_words(8, nb * words)
    y[: words] = 0
    z = np.zeros_like(x)
    assert (gpu_extract(plan, z, y, nb) == 0).all()
    got = gpu_extract(plan, x, y, nb)
    assert bits_at(got, 0, q) == 0
    assert (got == oracle_extract(plan, x, y, nb)).all()
    one = gpu_extract(plan, x[:words], y[:words], 1)
    assert (one == oracle_extract(plan, x[:words], y[:words], 1)).all()
    qext.qext_extract(plan, dev_words(x), dev_words(y), 0, dev_words(np.zeros(1, np.uint32)))
    # all-ones sources
    ones = np.full(nb * words, 0xFFFFFFFF, np.uint32)
    assert (gpu_extract(plan, ones, ones, nb) == oracle_extract(plan, ones, ones, nb)).all()


@pytest.mark.parametrize("b,ns,off", [(8, 4096, 0), (8, 4099, 0), (12, 1001, 0), (12, 8, 0), (12, 100003, 0),
                                      (16, 33, 0), (1, 999, 0), (5, 77, 0), (3, 1, 0), (11, 640, 0),
                                      (12, 1001, 1), (8, 333, 3), (16, 65, 1)])
def test_pack_matches_oracle(b, ns, off):
    """Vectorised paths (b = 8, 12, 16 on 16-byte aligned samples), their
    ragged tails, and the generic path (other b, or unaligned samples)."""
    s = workloads.adc_samples(b * 7 + ns, ns, b)
    s = s | np.uint16(0xFFFF ^ ((1 << b) - 1)) if b < 16 else s   # garbage above b must be ignored
    buf = torch.zeros(ns + off, dtype=torch.int16, device="cuda")
    buf[off:] = torch.from_numpy(s.view(np.int16)).cuda()
    ts = buf[off:]
    nw = -(-ns * b // 32)
    out = torch.full((nw + 4,), -1, dtype=torch.int32, device="cuda")
    qext.qext_pack_samples(b, ts, ns, out)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[nw:] == 0xFFFFFFFF).all()
    want = oracle.pack_samples(b, s & np.uint16((1 << b) - 1))
    assert (got[:nw] == want).all()


def test_config_plain_small_end_to_end():
    """4096 blocks x 256 bits, 8-bit ADC, seeds 0/1: GPU ingest + extraction
    against the oracle's ingest + extraction, every output bit."""
    spec = workloads.config_plain_small()
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    info = plan.info
    assert (info["q"], info["n_p"]) == (4, 64)
    sx, sy = spec.samples("x"), spec.samples("y")
    words = spec.nbits // 32
    px = torch.empty(words, dtype=torch.int32, device="cuda")
    py = torch.empty(words, dtype=torch.int32, device="cuda")
    qext.qext_pack_samples(spec.b, torch.from_numpy(sx.view(np.int16)).cuda(), sx.size, px)
    qext.qext_pack_samples(spec.b, torch.from_numpy(sy.view(np.int16)).cuda(), sy.size, py)
    out = torch.empty(spec.nblocks * info["m"] // 32, dtype=torch.int32, device="cuda")
    qext.qext_extract(plan, px, py, spec.nblocks, out)
    torch.cuda.synchronize()
    poly, _ = oracle.select_poly(info["q"])
    ox, oy = oracle.pack_samples(spec.b, sx), oracle.pack_samples(spec.b, sy)
    want = oracle.extract(info["q"], info["n_p"], info["m"], poly, ox, oy, spec.nblocks)
    assert want.size * 32 == spec.nblocks * info["q"] == spec.nbits // info["n_p"]   # Theorem 3.4
    assert (host_words(out) == want).all()


def test_config_large_single_stream_sampled():
    """2^20 blocks x 1024 bits (12-bit ADC, bias offset): the full-size launch,
    checked on sampled blocks (each recomputed by the oracle alone) and on the
    output length."""
    spec = workloads.config_large_single()
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    info = plan.info
    assert (info["q"], info["n_p"], info["m"]) == (16, 64, 16)
    words = spec.nbits // 32
    out_words = spec.nblocks * info["m"] // 32
    sx, sy = spec.samples("x"), spec.samples("y")
    px = torch.empty(-(-sx.size * 12 // 32), dtype=torch.int32, device="cuda")
    py = torch.empty_like(px)
    qext.qext_pack_samples(12, torch.from_numpy(sx.view(np.int16)).cuda(), sx.size, px)
    qext.qext_pack_samples(12, torch.from_numpy(sy.view(np.int16)).cuda(), sy.size, py)
    out = torch.full((out_words + 4,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract(plan, px, py, spec.nblocks, out)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[out_words:] == 0xFFFFFFFF).all()
    ox = oracle.pack_samples(12, sx)[:words]
    oy = oracle.pack_samples(12, sy)[:words]
    assert (host_words(px)[:words] == ox).all() and (host_words(py)[:words] == oy).all()
    rng = np.random.Generator(np.random.PCG64(99))
    sample = np.unique(np.concatenate([rng.integers(0, spec.nblocks, 3000), np.arange(40),
                                       np.arange(spec.nblocks - 40, spec.nblocks)]))
    poly, _ = oracle.select_poly(16)
    wpb = spec.n // 32
    for l in sample:
        l = int(l)
        z = oracle.extract(16, 64, 16, poly, ox[l * wpb:(l + 1) * wpb], oy[l * wpb:(l + 1) * wpb], 1)
        assert bits_at(got, l * 16, 16) == int(z[0]), "block %d" % l


SAMPLE_FLAGS = [0, qext.QEXT_F_RAW_PREFETCH, qext.QEXT_F_CTA_TILES,
                qext.QEXT_F_CTA_TILES | qext.QEXT_F_RAW_PREFETCH, qext.QEXT_F_WARP_SPECIALIZED]
SAMPLE_FLAG_IDS = ["warp_pipelines", "warp_pipelines_2buf", "cta_tiles", "cta_tiles_2buf", "warp_specialized"]


@pytest.mark.parametrize("q,b,nblocks,extra", [
    (16, 12, 1000, 0), (16, 12, 4133, 5), (16, 12, 129, 1), (4, 8, 4099, 0), (4, 12, 777, 3), (4, 16, 64, 0),
    (64, 12, 300, 1), (64, 16, 129, 0), (64, 8, 33, 2), (16, 8, 257, 0), (16, 16, 100, 7), (16, 12, 1, 0),
])
@pytest.mark.parametrize("flags", SAMPLE_FLAGS, ids=SAMPLE_FLAG_IDS)
def test_extract_samples_matches_oracle(q, b, nblocks, extra, flags):
    """Fused ingest + extraction from raw b-bit samples (garbage above b) against
    the oracle's packing followed by its extraction, every output bit."""
    plan = plan_for(q, 64)
    n = 64 * q
    ns = -(-nblocks * n // b) + extra
    s_x = workloads.adc_samples(q * 10 + b, ns, b, offset_amp=0.05)
    s_y = workloads.adc_samples(q * 10 + b + 1, ns, b, offset_amp=0.05)
    junk = np.uint16(0xFFFF ^ ((1 << b) - 1)) if b < 16 else np.uint16(0)
    gx = torch.from_numpy((s_x | junk).view(np.int16)).cuda()
    gy = torch.from_numpy((s_y | junk).view(np.int16)).cuda()
    nout = -(-nblocks * q // 32)
    out = torch.full((nout + 4,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract_samples_ex(plan, b, gx, gy, ns, nblocks, out, None, flags)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[nout:] == 0xFFFFFFFF).all()
    words = nblocks * n // 32
    ox = oracle.pack_samples(b, s_x)[:words]
    oy = oracle.pack_samples(b, s_y)[:words]
    want = oracle_extract(plan, ox, oy, nblocks)
    assert (got[:nout] == want).all()


@pytest.mark.parametrize("q,b,nblocks", [(16, 12, 200037), (4, 8, 600001), (16, 16, 150011)])
@pytest.mark.parametrize("flags", SAMPLE_FLAGS, ids=SAMPLE_FLAG_IDS)
def test_extract_samples_many_tiles_per_cta(q, b, nblocks, flags):
    """Enough tiles that every persistent CTA walks several of them (buffer
    reuse, raw-tile prefetch, the ragged last tile), every output bit."""
    plan = plan_for(q, 64)
    n = 64 * q
    ns = -(-nblocks * n // b)
    s_x = workloads.adc_samples(1000 + q + b, ns, b)
    s_y = workloads.adc_samples(2000 + q + b, ns, b)
    nout = -(-nblocks * q // 32)
    out = torch.full((nout + 4,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract_samples_ex(plan, b, torch.from_numpy(s_x.view(np.int16)).cuda(),
                                 torch.from_numpy(s_y.view(np.int16)).cuda(), ns, nblocks, out, None, flags)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[nout:] == 0xFFFFFFFF).all()
    words = nblocks * n // 32
    want = oracle_extract(plan, oracle.pack_samples(b, s_x)[:words], oracle.pack_samples(b, s_y)[:words], nblocks)
    assert (got[:nout] == want).all()


def test_extract_samples_rejects_short_input():
    plan = plan_for(16, 64)
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract_samples(plan, 12, 16, 16, 85, 1, 16)   # 85 samples < one 1024-bit block
    assert e.value.code == qext.QEXT_E_INVAL
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract_samples(plan, 10, 16, 16, 1000, 1, 16)
    assert e.value.code == qext.QEXT_E_UNSUPPORTED


@pytest.mark.parametrize("flags", SAMPLE_FLAGS[:4], ids=SAMPLE_FLAG_IDS[:4])
def test_config_large_single_stream_fused_sampled(flags):
    """2^20 blocks x 1024 bits from 12-bit samples through the fused path
    (the benchmark's launch), checked on sampled blocks against the oracle."""
    spec = workloads.config_large_single()
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    sx, sy = spec.samples("x"), spec.samples("y")
    out_words = spec.nblocks * 16 // 32
    out = torch.full((out_words + 4,), -1, dtype=torch.int32, device="cuda")
    qext.qext_extract_samples_ex(plan, 12, torch.from_numpy(sx.view(np.int16)).cuda(),
                                 torch.from_numpy(sy.view(np.int16)).cuda(), sx.size, spec.nblocks, out, None, flags)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[out_words:] == 0xFFFFFFFF).all()
    words = spec.nbits // 32
    ox = oracle.pack_samples(12, sx)[:words]
    oy = oracle.pack_samples(12, sy)[:words]
    rng = np.random.Generator(np.random.PCG64(7))
    sample = np.unique(np.concatenate([rng.integers(0, spec.nblocks, 3000), np.arange(40),
                                       np.arange(spec.nblocks - 40, spec.nblocks)]))
    poly, _ = oracle.select_poly(16)
    for l in sample:
        l = int(l)
        z = oracle.extract(16, 64, 16, poly, ox[l * 32:(l + 1) * 32], oy[l * 32:(l + 1) * 32], 1)
        assert bits_at(got, l * 16, 16) == int(z[0]), "block %d" % l


@pytest.mark.parametrize("q,b,nblocks,chunk", [(16, 12, 5000, 700), (16, 0, 3001, 512), (4, 8, 9000, 1000),
                                               (64, 12, 400, 100), (64, 0, 257, 64), (16, 16, 100, 1000)])
def test_pipeline_host_to_host_matches_oracle(q, b, nblocks, chunk):
    """qext_pipeline_run from pinned host buffers, chunked and overlapped,
    against the oracle (the benchmark's end-to-end path)."""
    plan = plan_for(q, 64)
    n = 64 * q
    pp = qext.qext_pipeline_create(plan, b, chunk)
    assert qext.qext_pipeline_info(pp)["chunk_blocks"] >= chunk
    if b:
        ns = -(-nblocks * n // b) + 3
        sx = workloads.adc_samples(b + q, ns, b)
        sy = workloads.adc_samples(b + q + 1, ns, b)
        hx = torch.from_numpy(sx.view(np.int16)).pin_memory()
        hy = torch.from_numpy(sy.view(np.int16)).pin_memory()
        count = ns
        ox = oracle.pack_samples(b, sx)[: nblocks * n // 32]
        oy = oracle.pack_samples(b, sy)[: nblocks * n // 32]
    else:
        ox = workloads.random_words(q + 5, nblocks * n // 32)
        oy = workloads.random_words(q + 6, nblocks * n // 32)
        hx = torch.from_numpy(ox.view(np.int32)).pin_memory()
        hy = torch.from_numpy(oy.view(np.int32)).pin_memory()
        count = nblocks * n
    nout = -(-nblocks * q // 32)
    out = torch.full((nout + 2,), -1, dtype=torch.int32).pin_memory()
    qext.qext_pipeline_run(pp, hx, hy, count, nblocks, out)
    got = out.numpy().view(np.uint32)
    assert (got[nout:] == 0xFFFFFFFF).all()
    assert (got[:nout] == oracle_extract(plan, ox, oy, nblocks)).all()
    pp.close()


@pytest.mark.parametrize("kernel", [0, qext.QEXT_F_CTA_TILES], ids=["per_warp_packed", "cta_tiles"])
def test_bounded_wait_times_out_and_context_survives(kernel):
    """Failure detection without a fault: the barrier is armed but no copy is
    issued, so every CTA's (per-warp kernel: every warp's) bounded wait runs
    out; the kernel records QEXT_E_TIMEOUT and returns, the host reads the
    status, and the next extraction on the same context is correct."""
    plan = plan_for(16, 64)
    nb = 4096
    x = workloads.random_words(71, nb * 32)
    y = workloads.random_words(72, nb * 32)
    tx, ty = dev_words(x), dev_words(y)
    out = torch.zeros(nb // 2, dtype=torch.int32, device="cuda")
    assert qext.qext_device_status() == qext.QEXT_OK
    qext.qext_extract_ex(plan, tx, ty, nb, out, None, qext.QEXT_F_TEST_TIMEOUT | kernel)
    torch.cuda.synchronize()
    assert qext.qext_device_status() == qext.QEXT_E_TIMEOUT
    assert qext.qext_device_status() == qext.QEXT_OK          # read clears it
    assert (gpu_extract(plan, x, y, nb) == oracle_extract(plan, x, y, nb)).all()
    assert qext.qext_device_status() == qext.QEXT_OK


def test_per_warp_bounded_wait_times_out_and_context_survives():
    """The same failure detection in the per-warp raw-sample kernel (the
    default of qext_extract_samples): each warp arms its barrier without a
    copy, gives up, records QEXT_E_TIMEOUT and returns; the next extraction on
    the same context is correct."""
    plan = plan_for(16, 64)
    nb = 6000
    ns = -(-nb * 1024 // 12)
    sx = workloads.adc_samples(81, ns, 12)
    sy = workloads.adc_samples(82, ns, 12)
    gx = torch.from_numpy(sx.view(np.int16)).cuda()
    gy = torch.from_numpy(sy.view(np.int16)).cuda()
    out = torch.zeros(nb // 2, dtype=torch.int32, device="cuda")
    assert qext.qext_device_status() == qext.QEXT_OK
    qext.qext_extract_samples_ex(plan, 12, gx, gy, ns, nb, out, None, qext.QEXT_F_TEST_TIMEOUT)
    torch.cuda.synchronize()
    assert qext.qext_device_status() == qext.QEXT_E_TIMEOUT
    assert qext.qext_device_status() == qext.QEXT_OK
    with pytest.raises(qext.QextError) as e:   # only the per-warp kernel has the test mode
        qext.qext_extract_samples_ex(plan, 12, gx, gy, ns, nb, out, None,
                                     qext.QEXT_F_TEST_TIMEOUT | qext.QEXT_F_CTA_TILES)
    assert e.value.code == qext.QEXT_E_INVAL
    qext.qext_extract_samples(plan, 12, gx, gy, ns, nb, out)
    torch.cuda.synchronize()
    words = nb * 32
    want = oracle_extract(plan, oracle.pack_samples(12, sx)[:words], oracle.pack_samples(12, sy)[:words], nb)
    assert (host_words(out) == want).all()
    assert qext.qext_device_status() == qext.QEXT_OK
