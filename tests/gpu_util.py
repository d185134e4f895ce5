"""Helpers for the GPU tests: move numpy words to the device and back, run
the C ABI, and compare with the oracle."""
import math

import numpy as np
import torch

import oracle
from paper_2402_14607_gb300 import qext


def dev_words(a: np.ndarray, pad_words: int = 0, offset_words: int = 0) -> torch.Tensor:
    """uint32 numpy words on cuda:0, optionally placed at a word offset
    inside a larger allocation (to exercise 4-byte-aligned pointers)."""
    a = np.ascontiguousarray(a, dtype=np.uint32)
    buf = torch.zeros(a.size + pad_words + offset_words, dtype=torch.int32, device="cuda")
    if a.size:
        buf[offset_words:offset_words + a.size] = torch.from_numpy(a.view(np.int32)).to("cuda")
    return buf[offset_words:]


def host_words(t: torch.Tensor) -> np.ndarray:
    return t.cpu().numpy().view(np.uint32)


def gpu_extract(plan, x: np.ndarray, y: np.ndarray, nblocks: int, offset_words: int = 0, flags: int = 0) -> np.ndarray:
    info = plan.info
    nout = -(-nblocks * info["m"] // 32)
    tx = dev_words(x, offset_words=offset_words)
    ty = dev_words(y, offset_words=offset_words)
    out = torch.full((nout + 8,), -1, dtype=torch.int32, device="cuda")  # sentinel past the end
    qext.qext_extract_ex(plan, tx, ty, nblocks, out, None, flags)
    torch.cuda.synchronize()
    res = host_words(out)
    assert (res[nout:] == 0xFFFFFFFF).all(), "kernel wrote past the output"
    return res[:nout]


def oracle_extract(plan, x, y, nblocks):
    info = plan.info
    poly, _ = oracle.select_poly(info["q"])
    return oracle.extract(info["q"], info["n_p"], info["m"], poly, x, y, nblocks)


def plan_for(q: int, n_p: int, m: int = 0):
    """A plan with exactly this (q, n_p), n_p >= 25.  k = n/2 + 12n/n_p makes
    Algorithm 1's ceil(24/(2 delta - 1)) equal n_p, so no larger q qualifies;
    eps is then any value above Theorem 3.1's bound for q."""
    n = q * n_p
    k = n / 2 + 12 * n / n_p
    l2 = oracle.log2_eps_block(n, k, q)
    if l2 >= math.log2(0.999):
        k = n - 0.25
        l2 = oracle.log2_eps_block(n, k, q)
    p = qext.qext_plan_create(n, m, k, min(0.999, 2.0 ** (l2 + 1e-3)))
    assert (p.info["q"], p.info["n_p"]) == (q, n_p), p.info
    return p


def bits_at(words: np.ndarray, start: int, count: int) -> int:
    w0 = start // 32
    w1 = (start + count + 31) // 32
    acc = 0
    for i, v in enumerate(words[w0:w1]):
        acc |= int(v) << (32 * i)
    return (acc >> (start - 32 * w0)) & ((1 << count) - 1)
