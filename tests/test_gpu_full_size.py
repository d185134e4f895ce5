"""Parity at the full sizes of the batched and sustained workloads, in the
launch configurations bench.py times, on sampled blocks that the oracle
computes one by one: the 64-stream batched launch (block counts up to 2^20,
n over {256, 1024, 4096}, 6.5 GB; random words, and 8- and 12-bit ADC samples
with their ingest in the same CUDA graph; inputs drawn on the device by
torch's seeded generator, the sampled blocks' bytes copied back for the
oracle), a full 256 MiB (2^31-bit) chunk of the sustained stream pushed after
a smaller one with state carried, and the sustained workload's raw-sample
chunks cycled as the benchmark pushes them."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.gpu_util import bits_at, host_words

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


def block_value(plan, xw: np.ndarray, yw: np.ndarray) -> int:
    info = plan.info
    poly, _ = oracle.select_poly(info["q"])
    z = oracle.extract(info["q"], info["n_p"], info["m"], poly, xw, yw, 1)
    return sum(int(w) << (32 * i) for i, w in enumerate(z))


def test_batched_full_size_sampled():
    specs = workloads.config_batched()
    gen = torch.Generator(device="cuda")
    gen.manual_seed(3)
    plans, items = {}, []
    for sp in specs:
        key = (sp.n, sp.k, sp.eps)
        if key not in plans:
            plans[key] = qext.qext_plan_create(sp.n, 0, sp.k, sp.eps)
        plan = plans[key]
        words = sp.nblocks * sp.n // 32
        x = torch.randint(-2 ** 31, 2 ** 31 - 1, (words,), dtype=torch.int32, device="cuda", generator=gen)
        y = torch.randint(-2 ** 31, 2 ** 31 - 1, (words,), dtype=torch.int32, device="cuda", generator=gen)
        out = torch.full((-(-sp.nblocks * plan.info["m"] // 32) + 1,), -1, dtype=torch.int32, device="cuda")
        items.append((plan, x, y, sp.nblocks, out))
    stream = torch.cuda.Stream()
    b = qext.qext_batch_create(items)
    qext.qext_batch_autotune(b, 1, stream)
    for it in items:
        it[4].fill_(-1)
    qext.qext_batch_capture(b, stream)
    qext.qext_batch_launch(b, stream)
    stream.synchronize()
    rng = np.random.Generator(np.random.PCG64(17))
    for (plan, x, y, nb, out), sp in zip(items, specs):
        got = host_words(out)
        m, wpb = plan.info["m"], sp.n // 32
        assert got[-1] == 0xFFFFFFFF, "wrote past the output"
        for l in np.unique(np.concatenate([rng.integers(0, nb, 3), [0, nb - 1]])):
            l = int(l)
            xw = host_words(x[l * wpb:(l + 1) * wpb])
            yw = host_words(y[l * wpb:(l + 1) * wpb])
            assert bits_at(got, l * m, m) == block_value(plan, xw, yw), (sp.n, nb, l)
    b.close()


def test_sustained_full_chunk_sampled():
    spec = workloads.config_sustained(total_bits=(1 << 24) + (1 << 31))
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    assert (plan.info["q"], plan.info["n_p"]) == (64, 64)
    sx, sy = spec.samples("x"), spec.samples("y")
    px = torch.empty(-(-sx.size * 12 // 32), dtype=torch.int32, device="cuda")
    py = torch.empty_like(px)
    qext.qext_pack_samples(12, torch.from_numpy(sx.view(np.int16)).cuda(), sx.size, px)
    qext.qext_pack_samples(12, torch.from_numpy(sy.view(np.int16)).cuda(), sy.size, py)
    s = qext.qext_stream_create(plan)
    outs = []
    w0 = 0
    for bits in (1 << 24, 1 << 31):   # a small chunk, then a full 256 MiB chunk, state carried
        out = torch.empty(bits // 4096 * 64 // 32, dtype=torch.int32, device="cuda")
        assert qext.qext_stream_push(s, px[w0:], py[w0:], bits, out, out.numel()) == out.numel()
        outs.append(out)
        w0 += bits // 32
    torch.cuda.synchronize()
    assert qext.qext_stream_info(s)["blocks_done"] == spec.nblocks
    s.close()
    got = np.concatenate([host_words(o) for o in outs])
    rng = np.random.Generator(np.random.PCG64(23))
    for l in np.unique(np.concatenate([rng.integers(0, spec.nblocks, 200), [0, 4095, 4096, spec.nblocks - 1]])):
        l = int(l)
        # block l's raw samples -> packed words by the oracle, from a sample
        # boundary at or before the block (1 sample = 12 bits)
        s0 = (4096 * l) // 12
        sh = 4096 * l - 12 * s0
        ox = oracle.pack_samples(12, sx[s0:s0 + 4096 // 12 + 2])
        oy = oracle.pack_samples(12, sy[s0:s0 + 4096 // 12 + 2])
        def cut(w):
            v = sum(int(a) << (32 * i) for i, a in enumerate(w)) >> sh
            return np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(128)], dtype=np.uint32)
        assert bits_at(got, l * 64, 64) == block_value(plan, cut(ox), cut(oy)), l


def test_sustained_raw_sample_chunks_full_size():
    """The sustained workload as the benchmark runs it: chunks of 178,956,288
    raw 12-bit samples (2^31 - 8192 bits, whole 3-block periods) with sigma
    drifting +-5 % over a 2^34-bit stream, two chunks per source cycled
    0, 1, 0 through qext_stream_push_samples (fused ingest, state carried);
    sampled blocks of every push, and its first and last blocks, match the
    oracle, and the repeated chunk gives the identical output."""
    chunk = 178956288
    total_bits = 1 << 34
    spec = workloads.config_sustained(total_bits=total_bits)
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    assert (plan.info["q"], plan.info["m"]) == (64, 64)
    nb = chunk * 12 // 4096
    hx, hy, gx, gy = [], [], [], []
    for c in range(2):
        kw = dict(drift_amp=0.05, drift_period=float(total_bits // 12), start=c * chunk)
        hx.append(workloads.adc_samples(spec.seed_x + 1000 * c, chunk, 12, **kw))
        hy.append(workloads.adc_samples(spec.seed_y + 1000 * c, chunk, 12, **kw))
        gx.append(torch.from_numpy(hx[-1].view(np.int16)).cuda())
        gy.append(torch.from_numpy(hy[-1].view(np.int16)).cuda())
    s = qext.qext_stream_create(plan)
    outs = []
    for c in (0, 1, 0):
        out = torch.empty(2 * nb, dtype=torch.int32, device="cuda")
        assert qext.qext_stream_push_samples(s, 12, gx[c], gy[c], chunk, out, 2 * nb) == 2 * nb
        outs.append(out)
    torch.cuda.synchronize()
    assert qext.qext_stream_info(s) == dict(blocks_done=3 * nb, tail_bits=0, pending_bits=0)
    s.close()
    assert torch.equal(outs[0], outs[2])
    poly, _ = oracle.select_poly(64)
    rng = np.random.Generator(np.random.PCG64(13))
    for c, out in ((0, outs[0]), (1, outs[1])):
        ox, oy = oracle.pack_samples(12, hx[c]), oracle.pack_samples(12, hy[c])
        got = host_words(out)
        for l in np.unique(np.concatenate([rng.integers(0, nb, 150), [0, 1, nb - 2, nb - 1]])):
            l = int(l)
            z = oracle.extract(64, 64, 64, poly, ox[l * 128:(l + 1) * 128], oy[l * 128:(l + 1) * 128], 1)
            assert int(got[2 * l]) == int(z[0]) and int(got[2 * l + 1]) == int(z[1]), "chunk %d block %d" % (c, l)


def _block_from_samples(plan, n, b, samples, l):
    """Oracle value of block l of a stream of b-bit samples (a device tensor):
    the samples around the block copied back, packed by the oracle and cut at
    the block's bit offset."""
    s0 = (n * l) // b
    sh = n * l - b * s0
    cnt = n // b + 2
    seg = samples[s0:s0 + cnt].cpu().numpy().view(np.uint16)
    w = oracle.pack_samples(b, seg)
    v = sum(int(a) << (32 * i) for i, a in enumerate(w)) >> sh
    words = np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(n // 32)], dtype=np.uint32)
    return words


def test_batched_adc_full_size_sampled():
    """The batched workload as the benchmark runs it: 64 stream pairs of 8- and
    12-bit ADC samples drawn on the device, the raw-sample batch (ingest inside
    the one batched launch) autotuned and replayed from its CUDA graph; sampled
    blocks of every stream (and its first and last) match the oracle, and the
    two-pass graph (every stream's ingest, then the packed-word batch) gives
    the same outputs."""
    specs = workloads.config_batched()
    plans, items, raw = {}, [], []
    for sp in specs:
        key = (sp.n, sp.k, sp.eps)
        if key not in plans:
            plans[key] = qext.qext_plan_create(sp.n, 0, sp.k, sp.eps)
        plan = plans[key]
        ns = -(-sp.nblocks * sp.n // sp.b)
        sx = workloads.adc_samples_device(sp.seed_x, ns, sp.b, "cuda")
        sy = workloads.adc_samples_device(sp.seed_y, ns, sp.b, "cuda")
        words = -(-ns * sp.b // 32)
        px = torch.empty(words, dtype=torch.int32, device="cuda")
        py = torch.empty_like(px)
        out = torch.full((-(-sp.nblocks * plan.info["m"] // 32) + 1,), -1, dtype=torch.int32, device="cuda")
        items.append((plan, px, py, sp.nblocks, out))
        raw.append((sp.b, sx, sy, ns))
    stream = torch.cuda.Stream()
    sh = int(stream.cuda_stream)
    bs = qext.qext_batch_create_samples([(plan, b_, sx, sy, ns, nb, out)
                                         for (b_, sx, sy, ns), (plan, _, _, nb, out) in zip(raw, items)])
    qext.qext_batch_autotune(bs, 1, stream)
    for it in items:
        it[4].fill_(-1)
    qext.qext_batch_capture(bs, stream)
    qext.qext_batch_launch(bs, stream)
    stream.synchronize()
    rng = np.random.Generator(np.random.PCG64(19))
    for (plan, _, _, nb, out), (b_, sx, sy, ns), sp in zip(items, raw, specs):
        got = host_words(out)
        m = plan.info["m"]
        assert got[-1] == 0xFFFFFFFF, "wrote past the output"
        for l in np.unique(np.concatenate([rng.integers(0, nb, 3), [0, nb - 1]])):
            l = int(l)
            xw = _block_from_samples(plan, sp.n, b_, sx, l)
            yw = _block_from_samples(plan, sp.n, b_, sy, l)
            assert bits_at(got, l * m, m) == block_value(plan, xw, yw), (sp.n, b_, nb, l)
    fused = [it[4].clone() for it in items]

    def ingest():
        for (b_, sx, sy, ns), (_, px, py, _, _) in zip(raw, items):
            qext.qext_pack_samples(b_, sx, ns, px, sh)
            qext.qext_pack_samples(b_, sy, ns, py, sh)

    ingest()
    b = qext.qext_batch_create(items)
    for it in items:
        it[4].fill_(-1)
    graph = torch.cuda.CUDAGraph()
    with torch.cuda.graph(graph, stream=stream):
        ingest()
        qext.qext_batch_run(b, sh)
    with torch.cuda.stream(stream):
        graph.replay()
    stream.synchronize()
    assert all(torch.equal(f, it[4]) for f, it in zip(fused, items))
    b.close()
    bs.close()
