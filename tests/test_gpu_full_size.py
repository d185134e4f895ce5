"""Parity at the full sizes of the batched and sustained workloads, in the
launch configurations bench.py times, on sampled blocks that the oracle
computes one by one: the 64-stream batched launch (block counts up to 2^20,
n over {256, 1024, 4096}, 6.5 GB; inputs drawn on the device by torch's
seeded generator, the sampled blocks' bytes copied back for the oracle) and a
full 256 MiB (2^31-bit) chunk of the sustained stream pushed after a smaller
one with state carried."""
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
