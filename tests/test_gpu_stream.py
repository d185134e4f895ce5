"""GPU tests of the stream-state manager (qext_stream_*): a stream pushed in
pieces of any bit length, with checkpoints in between, yields exactly the
oracle's one-shot output of Algorithm 1 on the whole stream (the blocks'
m-bit outputs concatenated in order; the final incomplete block dropped)."""
import numpy as np
import pytest
import torch

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext, workloads
from tests.gpu_util import bits_at, host_words, oracle_extract, plan_for

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    oracle.build()


def to_int(words):
    acc = 0
    for i, v in enumerate(np.asarray(words, dtype=np.uint32)):
        acc |= int(v) << (32 * i)
    return acc


def chunk_words(stream_int, a, L, offset_words=0, pad_garbage=True):
    """Device words holding stream bits [a, a+L), placed offset_words into a
    larger allocation; bits past L in the last word are garbage."""
    nw = (L + 31) // 32
    v = (stream_int >> a) & ((1 << L) - 1)
    if pad_garbage and L % 32:
        v |= (0x5A5A5A5A5A5A5A5A & ((1 << (32 * nw)) - 1)) & ~((1 << L) - 1)
    words = np.array([(v >> (32 * i)) & 0xFFFFFFFF for i in range(nw)], dtype=np.uint32)
    buf = torch.zeros(nw + offset_words + 1, dtype=torch.int32, device="cuda")
    if nw:
        buf[offset_words:offset_words + nw] = torch.from_numpy(words.view(np.int32)).cuda()
    return buf[offset_words:]


def run_stream(plan, xi, yi, splits, offsets=(0,), save_every=0):
    info = plan.info
    n, m = info["n"], info["m"]
    s = qext.qext_stream_create(plan)
    out_bits = 0
    nout = 0
    a = 0
    for idx, L in enumerate(splits):
        off = offsets[idx % len(offsets)]
        cx = chunk_words(xi, a, L, off)
        cy = chunk_words(yi, a, L, off)
        st = qext.qext_stream_info(s)
        newb = (st["tail_bits"] + L) // n
        cap = (st["pending_bits"] + newb * m + 31) // 32
        out = torch.full((cap + 2,), -1, dtype=torch.int32, device="cuda")
        w = qext.qext_stream_push(s, cx, cy, L, out, cap)
        torch.cuda.synchronize()
        got = host_words(out)
        assert (got[cap:] == 0xFFFFFFFF).all(), "push wrote past its capacity"
        out_bits |= to_int(got[:w]) << nout
        nout += 32 * w
        a += L
        if save_every and (idx + 1) % save_every == 0:
            state = qext.qext_stream_save(s)
            s.close()
            s = qext.qext_stream_restore(plan, state)
    out = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    fb = qext.qext_stream_flush(s, out, 1)
    torch.cuda.synchronize()
    if fb:
        last = int(host_words(out)[0])
        assert last >> fb == 0
        out_bits |= last << nout
        nout += fb
    info_s = qext.qext_stream_info(s)
    s.close()
    return out_bits, nout, info_s


def oracle_bits(plan, x, y, total_bits):
    info = plan.info
    nb = total_bits // info["n"]
    if nb == 0:
        return 0, 0
    want = oracle_extract(plan, x, y, nb)
    return to_int(want), nb * info["m"]


def random_splits(rng, total, n):
    splits = []
    left = total
    kinds = ["tiny", "sub", "block", "multi", "zero", "word"]
    while left > 0:
        k = kinds[int(rng.integers(len(kinds)))]
        if k == "tiny":
            L = int(rng.integers(1, 40))
        elif k == "sub":
            L = int(rng.integers(1, n))
        elif k == "block":
            L = n
        elif k == "multi":
            L = int(rng.integers(n, 7 * n))
        elif k == "word":
            L = 32 * int(rng.integers(1, 3 * n // 32))
        else:
            L = 0
        L = min(L, left)
        splits.append(L)
        left -= L
    return splits


@pytest.mark.parametrize("q,m,nblocks,seed", [
    (16, 16, 200, 1), (16, 13, 150, 2), (4, 4, 600, 3), (4, 3, 500, 4), (64, 64, 60, 5), (64, 41, 50, 6),
    (8, 8, 300, 7), (32, 17, 90, 8), (2, 1, 700, 9),
])
def test_split_invariance(q, m, nblocks, seed):
    """Arbitrary splits (zero-length, sub-block, misaligned bit lengths, 4-byte
    aligned pointers) give the one-shot output; the final partial block is
    dropped and the pending output bits come out on flush."""
    plan = plan_for(q, 64, m)
    n = 64 * q
    total = nblocks * n + 77
    rng = np.random.Generator(np.random.PCG64(seed))
    x = workloads.random_words(seed * 2, total // 32 + 2)
    y = workloads.random_words(seed * 2 + 1, total // 32 + 2)
    xi, yi = to_int(x), to_int(y)
    splits = random_splits(rng, total, n)
    got, nbits, st = run_stream(plan, xi, yi, splits, offsets=(0, 1, 3, 2))
    want, wbits = oracle_bits(plan, x, y, total)
    assert nbits == wbits == (total // n) * m        # Theorem 3.4: m * floor(L / n) bits
    assert got == want
    assert st["blocks_done"] == total // n


@pytest.mark.parametrize("q,m", [(16, 16), (16, 11), (64, 64), (4, 4)])
def test_save_restore_mid_stream(q, m):
    plan = plan_for(q, 64, m)
    n = 64 * q
    total = 120 * n + 5
    x = workloads.random_words(31, total // 32 + 2)
    y = workloads.random_words(32, total // 32 + 2)
    rng = np.random.Generator(np.random.PCG64(33))
    splits = random_splits(rng, total, n)
    got, nbits, _ = run_stream(plan, to_int(x), to_int(y), splits, offsets=(0, 1), save_every=3)
    want, wbits = oracle_bits(plan, x, y, total)
    assert nbits == wbits and got == want


def test_restore_rejects_other_plan():
    p16 = plan_for(16, 64)
    p4 = plan_for(4, 64)
    s = qext.qext_stream_create(p16)
    state = qext.qext_stream_save(s)
    with pytest.raises(qext.QextError) as e:
        qext.qext_stream_restore(p4, state)
    assert e.value.code == qext.QEXT_E_STATE
    with pytest.raises(qext.QextError) as e:
        qext.qext_stream_restore(p16, b"\0" * len(state))
    assert e.value.code == qext.QEXT_E_INVAL
    s.close()


def test_push_capacity_check():
    plan = plan_for(16, 64)
    s = qext.qext_stream_create(plan)
    x = torch.zeros(64, dtype=torch.int32, device="cuda")
    out = torch.zeros(1, dtype=torch.int32, device="cuda")
    with pytest.raises(qext.QextError) as e:
        qext.qext_stream_push(s, x, x, 2048, out, 0)     # two blocks need one word
    assert e.value.code == qext.QEXT_E_NOSPACE
    assert qext.qext_stream_info(s) == dict(blocks_done=0, tail_bits=0, pending_bits=0)
    s.close()


def test_sustained_chunks_fast_path():
    """Sustained-stream shape, scaled down: n = 4096, 12-bit ADC with sigma
    drifting +-5%, pushed in whole-block 16-byte-aligned chunks (the in-place
    path), state carried; sampled blocks checked against the oracle."""
    spec = workloads.config_sustained(total_bits=1 << 27)
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    info = plan.info
    assert (info["q"], info["n_p"]) == (64, 64)
    sx, sy = spec.samples("x"), spec.samples("y")
    px = torch.empty(-(-sx.size * 12 // 32), dtype=torch.int32, device="cuda")
    py = torch.empty_like(px)
    qext.qext_pack_samples(12, torch.from_numpy(sx.view(np.int16)).cuda(), sx.size, px)
    qext.qext_pack_samples(12, torch.from_numpy(sy.view(np.int16)).cuda(), sy.size, py)
    chunk_bits = 1 << 24
    s = qext.qext_stream_create(plan)
    outs = []
    for c in range(spec.nbits // chunk_bits):
        w0 = c * chunk_bits // 32
        out = torch.empty(chunk_bits // 4096 * 64 // 32, dtype=torch.int32, device="cuda")
        w = qext.qext_stream_push(s, px[w0:], py[w0:], chunk_bits, out, out.numel())
        assert w == out.numel()
        outs.append(out)
    torch.cuda.synchronize()
    got = np.concatenate([host_words(o) for o in outs])
    assert qext.qext_stream_info(s)["blocks_done"] == spec.nblocks
    s.close()
    ox = oracle.pack_samples(12, sx)
    oy = oracle.pack_samples(12, sy)
    assert (host_words(px)[:spec.nbits // 32] == ox[:spec.nbits // 32]).all()
    rng = np.random.Generator(np.random.PCG64(5))
    poly, _ = oracle.select_poly(64)
    for l in np.unique(np.concatenate([rng.integers(0, spec.nblocks, 300), [0, spec.nblocks - 1]])):
        l = int(l)
        z = oracle.extract(64, 64, 64, poly, ox[l * 128:(l + 1) * 128], oy[l * 128:(l + 1) * 128], 1)
        assert bits_at(got, l * 64, 64) == int(z[0]) | (int(z[1]) << 32), "block %d" % l


def _push_raw(s, plan, b, sx, sy, a, k, misalign):
    """Push samples [a, a + k) of each source as a fresh device array (16-byte
    aligned, or 2-byte aligned with misalign); returns the output words."""
    info = plan.info
    st = qext.qext_stream_info(s)
    newb = (st["tail_bits"] + k * b) // info["n"]
    cap = (st["pending_bits"] + newb * info["m"] + 31) // 32
    out = torch.full((cap + 2,), -1, dtype=torch.int32, device="cuda")
    off = 1 if misalign else 0
    gx = torch.zeros(k + off + 8, dtype=torch.int16, device="cuda")
    gy = torch.zeros_like(gx)
    if k:
        gx[off:off + k] = torch.from_numpy(sx[a:a + k].view(np.int16)).cuda()
        gy[off:off + k] = torch.from_numpy(sy[a:a + k].view(np.int16)).cuda()
    w = qext.qext_stream_push_samples(s, b, gx[off:], gy[off:], k, out, cap)
    torch.cuda.synchronize()
    got = host_words(out)
    assert (got[cap:] == 0xFFFFFFFF).all(), "push wrote past its capacity"
    return got[:w]


def _realigning_count(plan, st, b, limit):
    """Smallest k <= limit after which the stream holds no tail and no pending bits."""
    n, m = plan.info["n"], plan.info["m"]
    for k in range(1, limit + 1):
        v = st["tail_bits"] + k * b
        if v % n == 0 and (st["pending_bits"] + (v // n) * m) % 32 == 0:
            return k
    return None


@pytest.mark.parametrize("q,m,b,seed", [(16, 16, 12, 1), (64, 64, 12, 2), (4, 4, 8, 3), (16, 13, 16, 4),
                                         (64, 41, 8, 5), (8, 8, 12, 6), (16, 16, 5, 7)])
def test_raw_sample_pushes_match_oracle(q, m, b, seed):
    """Raw-sample pushes (qext_stream_push_samples) of random sample counts,
    some starting on a block boundary with nothing pending (fused path), some
    not (packed into the stream's staging buffers), mixed with pushes of the
    packed bits and a checkpoint, give the oracle's one-shot output of the
    whole stream."""
    plan = plan_for(q, 64, m)
    info = plan.info
    n = info["n"]
    rng = np.random.Generator(np.random.PCG64(seed))
    total = 60 * n // b + 3
    sx = workloads.adc_samples(100 + seed, total, b)
    sy = workloads.adc_samples(200 + seed, total, b)
    ox, oy = oracle.pack_samples(b, sx), oracle.pack_samples(b, sy)
    xi, yi = to_int(ox), to_int(oy)
    s = qext.qext_stream_create(plan)
    out_bits, nout, a, step = 0, 0, 0, 0
    while a < total:
        st = qext.qext_stream_info(s)
        kind = step % 5
        if kind == 0:                      # realign, then a whole-period push (fused where supported)
            k = _realigning_count(plan, st, b, total - a) or (total - a)
        elif kind == 3:                    # packed bits of the next samples (qext_stream_push)
            k = min(int(rng.integers(1, 3 * n // b)), total - a)
        else:
            k = min(int(rng.integers(0, 4 * n // b)), total - a)
        if kind == 3:
            L = k * b
            cx, cy = chunk_words(xi, a * b, L), chunk_words(yi, a * b, L)
            newb = (st["tail_bits"] + L) // n
            cap = (st["pending_bits"] + newb * info["m"] + 31) // 32
            out = torch.full((cap + 2,), -1, dtype=torch.int32, device="cuda")
            w = qext.qext_stream_push(s, cx, cy, L, out, cap)
            torch.cuda.synchronize()
            words = host_words(out)[:w]
        else:
            words = _push_raw(s, plan, b, sx, sy, a, k, misalign=(kind == 4))
        out_bits |= to_int(words) << nout
        nout += 32 * len(words)
        a += k
        step += 1
        if step == 7:
            state = qext.qext_stream_save(s)
            s.close()
            s = qext.qext_stream_restore(plan, state)
    out = torch.full((2,), -1, dtype=torch.int32, device="cuda")
    fb = qext.qext_stream_flush(s, out, 1)
    torch.cuda.synchronize()
    if fb:
        out_bits |= int(host_words(out)[0]) << nout
        nout += fb
    s.close()
    want, wbits = oracle_bits(plan, ox, oy, total * b)
    assert nout == wbits
    assert out_bits == want


def test_raw_sample_full_chunk_with_carried_state():
    """The sustained workload's chunk at full size: 12-bit samples with drifting
    sigma, n = 4096.  A small whole-period push (fused path), then 1000 samples
    that end mid-block, then one full chunk of 178,956,288 samples (2^31 - 8192
    bits: the largest whole number of 3-block periods within 256 MiB) pushed
    with that tail carried, then a realigning push; sampled blocks of every
    part, and the blocks around each boundary, match the oracle."""
    chunk = 178956288
    first, mid = 1024, 1000
    spec = workloads.config_sustained(total_bits=(first + mid + chunk + 4096) * 12)
    plan = qext.qext_plan_create(spec.n, 0, spec.k, spec.eps)
    assert (plan.info["q"], plan.info["m"]) == (64, 64)
    sx, sy = spec.samples("x"), spec.samples("y")
    gx = torch.from_numpy(sx.view(np.int16)).cuda()
    gy = torch.from_numpy(sy.view(np.int16)).cuda()
    s = qext.qext_stream_create(plan)
    parts = []
    a = 0
    for k in (first, mid, chunk):
        st = qext.qext_stream_info(s)
        cap = (st["pending_bits"] + (st["tail_bits"] + 12 * k) // 4096 * 64 + 31) // 32
        out = torch.empty(cap + 1, dtype=torch.int32, device="cuda")
        w = qext.qext_stream_push_samples(s, 12, gx[a:], gy[a:], k, out, cap)
        parts.append(out[:w])
        a += k
    st = qext.qext_stream_info(s)
    k = _realigning_count(plan, st, 12, 4096)
    cap = (st["tail_bits"] + 12 * k) // 4096 * 2
    out = torch.empty(cap + 1, dtype=torch.int32, device="cuda")
    parts.append(out[:qext.qext_stream_push_samples(s, 12, gx[a:], gy[a:], k, out, cap)])
    a += k
    torch.cuda.synchronize()
    got = np.concatenate([host_words(p) for p in parts])
    nb = a * 12 // 4096
    assert qext.qext_stream_info(s) == dict(blocks_done=nb, tail_bits=0, pending_bits=0)
    s.close()
    assert got.size == 2 * nb
    ox = oracle.pack_samples(12, sx[:a])
    oy = oracle.pack_samples(12, sy[:a])
    poly, _ = oracle.select_poly(64)
    b1 = first * 12 // 4096
    b2 = (first + mid) * 12 // 4096
    rng = np.random.Generator(np.random.PCG64(11))
    sample = np.unique(np.concatenate([rng.integers(0, nb, 300), np.arange(0, 6), np.arange(b1 - 2, b2 + 3),
                                       np.arange(nb - 6, nb)]))
    for l in sample:
        l = int(l)
        z = oracle.extract(64, 64, 64, poly, ox[l * 128:(l + 1) * 128], oy[l * 128:(l + 1) * 128], 1)
        assert bits_at(got, l * 64, 64) == int(z[0]) | (int(z[1]) << 32), "block %d" % l
