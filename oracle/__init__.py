"""CPU oracle for Ext_bs^eq (Algorithm 1) of arXiv 2402.14607.

TEST INFRASTRUCTURE ONLY: the tests, ``__graft_entry__.smoke()`` and the CPU
baseline of ``bench.py`` may import this package; the library under
``paper_2402_14607_gb300`` never does.  The arithmetic lives in the plain C
file ``qext_oracle.c`` (bit-serial GF(2^q) multiply, Rabin irreducibility
test, Algorithm 1 block loop); this module compiles it with gcc and wraps it
with ctypes.  It shares no code with the CUDA path.

Every routine cites the passage it follows:
  gf_mul            -- Sec. 3.2, multiplication in F_{2^q} (bit-serial).
  select_poly       -- Sec. 3.2 leaves P_q open; minimum-weight,
                       lexicographically first irreducible polynomial.
  ext_ip            -- Definition 3.2, Ext_IP^{n,q}(x,y) = sum_i x_i y_i.
  extract           -- Algorithm 1 (Ext_bs^eq), output truncated to m bits.
  plan              -- Definition 2.3 arguments, Algorithm 1's n, Theorem 3.1.
  alg1_params       -- Algorithm 1's parameter line (n and q from b,N,delta,eps).
  log2_eps_block    -- Theorem 3.1's per-block error.
  pack_samples      -- Sec. 3: X = X_1...X_N in ({0,1}^b)^N, LSB-first packing.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "qext_oracle.c")
_BUILD = os.path.join(_HERE, "_build")
_LIB = os.path.join(_BUILD, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile qext_oracle.c into oracle/_build/liboracle.so (gcc -O2, OpenMP
    when the host compiler has it).  Returns the library path."""
    with _lock:
        if (not force and os.path.exists(_LIB)
                and os.path.getmtime(_LIB) >= os.path.getmtime(_SRC)):
            return _LIB
        os.makedirs(_BUILD, exist_ok=True)
        tmp = _LIB + ".tmp%d" % os.getpid()
        base = ["gcc", "-O2", "-std=c11", "-shared", "-fPIC", _SRC, "-o", tmp, "-lm"]
        r = subprocess.run(base[:2] + ["-fopenmp"] + base[2:], capture_output=True, text=True)
        if r.returncode != 0:
            r = subprocess.run(base, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError("oracle build failed:\n" + r.stderr)
        os.replace(tmp, _LIB)
        return _LIB


def _load():
    global _lib
    if _lib is None:
        _lib = _configure(ctypes.CDLL(build()))
    return _lib


def _configure(lib):
    """Declare the C signatures on a loaded oracle library."""
    u64p = ctypes.POINTER(ctypes.c_uint64)
    u32p = ctypes.POINTER(ctypes.c_uint32)
    intp = ctypes.POINTER(ctypes.c_int)
    lib.orc_gf_mul.argtypes = [ctypes.c_int, u64p, u64p, u64p, u64p]
    lib.orc_gf_mul.restype = None
    lib.orc_is_irreducible.argtypes = [ctypes.c_int, u64p]
    lib.orc_is_irreducible.restype = ctypes.c_int
    lib.orc_select_poly.argtypes = [ctypes.c_int, u64p, intp]
    lib.orc_select_poly.restype = ctypes.c_int
    lib.orc_ext_ip.argtypes = [ctypes.c_int, ctypes.c_int, u64p, u64p, u64p, u64p]
    lib.orc_ext_ip.restype = None
    lib.orc_extract.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, u64p, u32p, u32p,
                                ctypes.c_uint64, u32p, ctypes.c_int]
    lib.orc_extract.restype = ctypes.c_int
    lib.orc_log2_eps_block.argtypes = [ctypes.c_uint32, ctypes.c_double, ctypes.c_uint32]
    lib.orc_log2_eps_block.restype = ctypes.c_double
    lib.orc_plan.argtypes = [ctypes.c_uint32, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                             u32p, u32p, u32p, ctypes.POINTER(ctypes.c_double)]
    lib.orc_plan.restype = ctypes.c_int
    lib.orc_alg1_params.argtypes = [ctypes.c_double, ctypes.c_uint32, ctypes.c_double, ctypes.c_double,
                                    u32p, u32p]
    lib.orc_alg1_params.restype = ctypes.c_int
    lib.orc_extract_alg2.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_int, u32p, u32p, u32p,
                                     ctypes.POINTER(ctypes.c_int)]
    lib.orc_extract_alg2.restype = ctypes.c_int
    lib.orc_alg2_log2_error.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    lib.orc_alg2_log2_error.restype = ctypes.c_double
    lib.orc_sample_histogram.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint16), ctypes.c_uint64, u64p]
    lib.orc_sample_histogram.restype = None
    lib.orc_min_entropy_estimate.argtypes = [ctypes.c_uint32, u64p]
    lib.orc_min_entropy_estimate.restype = ctypes.c_double
    lib.orc_pack_samples.argtypes = [ctypes.c_uint32, ctypes.POINTER(ctypes.c_uint16), ctypes.c_uint64, u32p]
    lib.orc_pack_samples.restype = None
    lib.orc_max_q.restype = ctypes.c_int
    lib.orc_has_openmp.restype = ctypes.c_int
    return lib


def _u64(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64))


def _u32(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_uint32))


def _words(v: int, nw: int) -> np.ndarray:
    return np.array([(v >> (64 * w)) & 0xFFFFFFFFFFFFFFFF for w in range(nw)], dtype=np.uint64)


def _int(a: np.ndarray) -> int:
    return sum(int(x) << (64 * i) for i, x in enumerate(a))


def max_q() -> int:
    return _load().orc_max_q()


def openmp_threads() -> int:
    """OpenMP thread count the oracle would use (0 if built without OpenMP)."""
    return _load().orc_has_openmp()


def gf_mul(q: int, poly: int, a: int, b: int) -> int:
    """a*b in F_2[alpha]/poly(alpha), poly given as an integer bit mask of
    degree q (bit d = coefficient of x^d); a, b < 2^q."""
    lib = _load()
    nw = q // 64 + 2
    ew = (q + 63) // 64
    out = np.zeros(nw, dtype=np.uint64)
    lib.orc_gf_mul(q, _u64(_words(poly, nw)), _u64(_words(a, nw)), _u64(_words(b, nw)), _u64(out))
    return _int(out[:ew])


def is_irreducible(q: int, poly: int) -> bool:
    """Rabin's test (degree-q polynomial given as an integer bit mask)."""
    return bool(_load().orc_is_irreducible(q, _u64(_words(poly, q // 64 + 2))))


def select_poly(q: int):
    """(poly_mask, taps) of the minimum-weight, lexicographically first
    irreducible polynomial of degree q; taps are the exponents strictly
    between 0 and q, descending."""
    lib = _load()
    out = np.zeros(q // 64 + 2, dtype=np.uint64)
    taps = (ctypes.c_int * 3)()
    w = lib.orc_select_poly(q, _u64(out), taps)
    if w == 0:
        raise ValueError("no irreducible trinomial/pentanomial of degree %d" % q)
    return _int(out), tuple(t for t in taps if t)


def ext_ip(q: int, poly: int, xs, ys) -> int:
    """Definition 3.2: sum_i xs[i]*ys[i] in GF(2^q) (elements as ints)."""
    lib = _load()
    ew = (q + 63) // 64
    n_p = len(xs)
    assert len(ys) == n_p
    xa = np.concatenate([_words(v, ew) for v in xs]) if n_p else np.zeros(0, np.uint64)
    ya = np.concatenate([_words(v, ew) for v in ys]) if n_p else np.zeros(0, np.uint64)
    out = np.zeros(ew, dtype=np.uint64)
    lib.orc_ext_ip(q, n_p, _u64(_words(poly, q // 64 + 2)), _u64(xa), _u64(ya), _u64(out))
    return _int(out)


def extract(q: int, n_p: int, m: int, poly: int, x: np.ndarray, y: np.ndarray, nblocks: int,
            threads: int = 0) -> np.ndarray:
    """Algorithm 1 over ``nblocks`` whole blocks of the packed uint32 streams
    x and y; returns ceil(nblocks*m/32) output words."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    need = (nblocks * q * n_p + 31) // 32
    if x.size < need or y.size < need:
        raise ValueError("streams shorter than nblocks blocks")
    out = np.zeros(max(1, (nblocks * m + 31) // 32), dtype=np.uint32)
    rc = lib.orc_extract(q, n_p, m, _u64(_words(poly, q // 64 + 2)), _u32(x), _u32(y), nblocks, _u32(out),
                         threads)
    if rc != 0:
        raise ValueError("orc_extract rejected its arguments (rc=%d)" % rc)
    return out[: (nblocks * m + 31) // 32]


def extract_alg2(n_p: int, q1: int, dq: int, nblocks: int, x: np.ndarray, y: np.ndarray,
                 taps=None) -> np.ndarray:
    """Algorithm 2 (Sec. 3.3) over its first ``nblocks`` blocks: block l has
    q_l = q1 + l*dq (dq = Delta*b) and takes the next q_l*n_p stream bits of
    each packed uint32 stream; returns the concatenated outputs (sum q_l bits)
    as uint32 words.  ``taps``: per block the taps (c, b, a) of P_{q_l} below
    x^{q_l} (0 past a trinomial's one tap), e.g. as select_poly found them
    earlier; None makes the oracle search every P_{q_l} itself."""
    lib = _load()
    x = np.ascontiguousarray(x, dtype=np.uint32)
    y = np.ascontiguousarray(y, dtype=np.uint32)
    qs = [q1 + l * dq for l in range(nblocks)]
    need = (n_p * sum(qs) + 31) // 32
    if x.size < need or y.size < need:
        raise ValueError("streams shorter than nblocks blocks")
    out = np.zeros(max(1, (sum(qs) + 31) // 32), dtype=np.uint32)
    tp = None
    if taps is not None:
        t = np.zeros(3 * nblocks, dtype=np.int32)
        for l in range(nblocks):
            for i, v in enumerate(list(taps[l])[:3]):
                t[3 * l + i] = int(v)
        tp = t.ctypes.data_as(ctypes.POINTER(ctypes.c_int))
    if lib.orc_extract_alg2(n_p, q1, dq, nblocks, _u32(x), _u32(y), _u32(out), tp) != 0:
        raise ValueError("bad Algorithm 2 parameters")
    return out


def alg2_log2_error(n_p: int, delta: float, q1: int, dq: int, nblocks: int) -> float:
    """log2 of Theorem 3.3's bound for the first nblocks outputs of Algorithm 2."""
    return _load().orc_alg2_log2_error(n_p, delta, q1, dq, nblocks)


def sample_histogram(b: int, samples: np.ndarray, counts: np.ndarray | None = None) -> np.ndarray:
    """counts[v] += #samples whose low b bits equal v (2^b uint64 counts)."""
    lib = _load()
    s = np.ascontiguousarray(samples, dtype=np.uint16)
    c = np.zeros(1 << b, dtype=np.uint64) if counts is None else counts
    lib.orc_sample_histogram(b, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), s.size, _u64(c))
    return c


def min_entropy_estimate(b: int, counts: np.ndarray) -> float:
    """Plug-in min-entropy -log2(max count / total) of a sample histogram."""
    return _load().orc_min_entropy_estimate(b, _u64(np.ascontiguousarray(counts, dtype=np.uint64)))


def log2_eps_block(n: int, k: float, q: int) -> float:
    return _load().orc_log2_eps_block(n, k, q)


class PlanError(ValueError):
    pass


def plan(n: int, m: int, k: float, eps: float):
    """Per-block plan; returns dict(n_p, q, m, log2_eps, poly, taps)."""
    lib = _load()
    n_p = ctypes.c_uint32()
    q = ctypes.c_uint32()
    mo = ctypes.c_uint32()
    le = ctypes.c_double()
    rc = lib.orc_plan(n, m, k, eps, ctypes.byref(n_p), ctypes.byref(q), ctypes.byref(mo), ctypes.byref(le))
    if rc != 0:
        raise PlanError({-1: "bad arguments", -2: "entropy rate <= 1/2",
                         -3: "no block factorisation meets eps"}[rc])
    poly, taps = select_poly(q.value)
    return dict(n=n, n_p=n_p.value, q=q.value, m=mo.value, log2_eps=le.value, poly=poly, taps=taps)


def alg1_params(N: float, b: int, delta: float, eps: float):
    lib = _load()
    n_p = ctypes.c_uint32()
    q = ctypes.c_uint32()
    rc = lib.orc_alg1_params(N, b, delta, eps, ctypes.byref(n_p), ctypes.byref(q))
    if rc != 0:
        raise PlanError("alg1_params rc=%d" % rc)
    return n_p.value, q.value


def pack_samples(b: int, samples: np.ndarray) -> np.ndarray:
    lib = _load()
    s = np.ascontiguousarray(samples, dtype=np.uint16)
    out = np.zeros(max(1, (s.size * b + 31) // 32), dtype=np.uint32)
    lib.orc_pack_samples(b, s.ctypes.data_as(ctypes.POINTER(ctypes.c_uint16)), s.size, _u32(out))
    return out[: (s.size * b + 31) // 32]


if __name__ == "__main__":  # pragma: no cover
    print(build(force="--force" in sys.argv))
