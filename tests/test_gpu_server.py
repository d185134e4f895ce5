"""Serving loop on the GPU: requests from many channels (different n, packed
or 12-bit sample input, whole or partial blocks) submitted together give, per
request, exactly the output they give alone, and per channel the oracle's
output of the concatenated stream; admission stays within the HBM budget."""
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


CHANNELS = [  # n, k, eps, b (0 = packed words)
    (1024, 867, 2.0 ** -50, 12), (256, 206, 2.0 ** -9, 12), (4096, 3485, 2.0 ** -52, 0), (1024, 867, 2.0 ** -50, 0),
    (256, 202, 2.0 ** -9, 0), (4096, 3485, 2.0 ** -52, 12),
]


def make_requests(seed):
    """Per channel: a raw stream (x, y) cut into requests of varied sizes."""
    rng = np.random.Generator(np.random.PCG64(seed))
    chans = []
    for ci, (n, k, eps, b) in enumerate(CHANNELS):
        reqs = []
        total = 0
        for r in range(4):
            whole = r % 2 == 0
            if b:
                ns = int(rng.integers(2, 40)) * n // 4 if whole else int(rng.integers(5, 40 * n // b))
                ns = ns if not whole else (ns * b // n) * n // b or n // 4
                count = ns
                bits = ns * b
            else:
                bits = int(rng.integers(1, 30)) * n if whole else int(rng.integers(1, 30 * n)) // 32 * 32 + 32
                count = bits
            reqs.append((count, bits))
            total += bits
        chans.append(dict(n=n, k=k, eps=eps, b=b, reqs=reqs, seed=seed * 100 + ci))
    for ch in chans:
        b = ch["b"]
        if b:
            ns = sum(c for c, _ in ch["reqs"])
            ch["sx"] = workloads.adc_samples(ch["seed"], ns, 12, offset_amp=0.05)
            ch["sy"] = workloads.adc_samples(ch["seed"] + 7, ns, 12, offset_amp=0.05)
        else:
            nw = sum(c // 32 for c, _ in ch["reqs"])
            ch["wx"] = workloads.random_words(ch["seed"], nw)
            ch["wy"] = workloads.random_words(ch["seed"] + 7, nw)
    return chans


def submit_channel(s, plans, ci, ch, outs):
    c = qext.qext_server_add_channel(s, plans[ci])
    off = 0
    rids = []
    for count, bits in ch["reqs"]:
        cap = (bits // ch["n"] + 2) * plans[ci].info["m"] // 32 + 2
        out = torch.full((cap,), -1, dtype=torch.int32).pin_memory()
        if ch["b"]:
            hx = torch.from_numpy(ch["sx"][off:off + count].view(np.int16).copy()).pin_memory()
            hy = torch.from_numpy(ch["sy"][off:off + count].view(np.int16).copy()).pin_memory()
            off += count
        else:
            w = count // 32
            hx = torch.from_numpy(ch["wx"][off:off + w].view(np.int32).copy()).pin_memory()
            hy = torch.from_numpy(ch["wy"][off:off + w].view(np.int32).copy()).pin_memory()
            off += w
        rid = qext.qext_server_submit(s, c, ch["b"], hx, hy, count, out, cap)
        outs[rid] = (ci, out)
        rids.append(rid)
    return rids


def collect(s, outs):
    qext.qext_server_drain(s, 120.0)
    done = qext.qext_server_poll(s, 10000)
    res = {}
    for d in done:
        assert d["status"] == qext.QEXT_OK, d
        ci, out = outs[d["request_id"]]
        words = out.numpy().view(np.uint32)
        res[d["request_id"]] = (ci, d, words[: -(-d["out_bits"] // 32)].copy())
    return res


def bits_of(words, nbits):
    acc = 0
    for i, v in enumerate(words):
        acc |= int(v) << (32 * i)
    return acc & ((1 << nbits) - 1)


def test_mix_equals_alone_and_oracle():
    chans = make_requests(5)
    plans = [qext.qext_plan_create(ch["n"], 0, ch["k"], ch["eps"]) for ch in chans]
    # all channels at once
    s = qext.qext_server_create(hbm_budget_bytes=256 << 20, max_batch=64)
    outs, mix_rids = {}, []
    for ci, ch in enumerate(chans):
        mix_rids.append(submit_channel(s, plans, ci, ch, outs))
    mix = collect(s, outs)
    st = qext.qext_server_get_stats(s)
    assert st["peak_bytes"] <= st["budget_bytes"]
    s.close()
    # each channel alone
    for ci, ch in enumerate(chans):
        s = qext.qext_server_create(hbm_budget_bytes=256 << 20, max_batch=64)
        outs_a = {}
        rids = submit_channel(s, plans, ci, ch, outs_a)
        alone = collect(s, outs_a)
        s.close()
        concat, nbits = 0, 0
        for r_mix, r_alone in zip(mix_rids[ci], rids):
            _, dm, wm = mix[r_mix]
            _, da, wa = alone[r_alone]
            assert dm["out_bits"] == da["out_bits"]
            assert bits_of(wm, dm["out_bits"]) == bits_of(wa, da["out_bits"]), (ci, r_mix)
            concat |= bits_of(wm, dm["out_bits"]) << nbits
            nbits += dm["out_bits"]
        # the channel's requests, concatenated, are Algorithm 1 on the whole stream
        info = plans[ci].info
        poly, _ = oracle.select_poly(info["q"])
        if ch["b"]:
            total_bits = len(ch["sx"]) * 12
            ox, oy = oracle.pack_samples(12, ch["sx"]), oracle.pack_samples(12, ch["sy"])
        else:
            total_bits = len(ch["wx"]) * 32
            ox, oy = ch["wx"], ch["wy"]
        nb = total_bits // ch["n"]
        want = oracle.extract(info["q"], info["n_p"], info["m"], poly, ox, oy, nb)
        assert nbits == nb * info["m"]
        assert concat == bits_of(want, nbits), ci


def test_tight_budget_queues_and_completes():
    chans = make_requests(6)
    plans = [qext.qext_plan_create(ch["n"], 0, ch["k"], ch["eps"]) for ch in chans]
    s = qext.qext_server_create(hbm_budget_bytes=4 << 20, max_batch=4)
    outs = {}
    for ci, ch in enumerate(chans):
        submit_channel(s, plans, ci, ch, outs)
    res = collect(s, outs)
    st = qext.qext_server_get_stats(s)
    assert len(res) == st["submitted"] == st["completed"]
    assert st["peak_bytes"] <= 4 << 20
    assert all(d["latency_s"] > 0 for _, d, _ in res.values())
    s.close()
