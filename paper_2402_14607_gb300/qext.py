"""Thin Python binding of libqext (include/qext.h): the same names, argument
marshalling only.  Every computation runs in the CUDA library; if the library
is not built this module raises instead of computing anything itself.

Pointers may be given as integers or as torch tensors (their data_ptr());
streams as None (torch's current stream), a torch.cuda.Stream, or an int
handle.
"""
from __future__ import annotations

import ctypes
import os

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_build", "libqext.so")

QEXT_OK = 0
QEXT_E_INVAL = -1
QEXT_E_ENTROPY = -2
QEXT_E_PARAM = -3
QEXT_E_UNSUPPORTED = -4
QEXT_E_CUDA = -5
QEXT_E_TIMEOUT = -6
QEXT_E_BUDGET = -7
QEXT_E_STATE = -8
QEXT_E_NOSPACE = -9
QEXT_E_LIMIT = -10
QEXT_NOALLOC_MAX_ITEMS = 1024
QEXT_F_DIRECT = 0x1
QEXT_F_NBUF1 = 0x2
QEXT_F_TILE32 = 0x4
QEXT_F_TILE64 = 0x8
QEXT_F_TEST_TIMEOUT = 0x10
QEXT_F_WARP_SPECIALIZED = 0x20
QEXT_F_RAW_PREFETCH = 0x40
QEXT_F_CTA_TILES = 0x80

_lib = None


class BatchItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("x", ctypes.c_void_p), ("y", ctypes.c_void_p),
                ("nblocks", ctypes.c_uint64), ("out", ctypes.c_void_p)]


class BatchSamplesItem(ctypes.Structure):
    _fields_ = [("plan", ctypes.c_void_p), ("b", ctypes.c_uint32), ("x_samples", ctypes.c_void_p),
                ("y_samples", ctypes.c_void_p), ("nsamples", ctypes.c_uint64), ("nblocks", ctypes.c_uint64),
                ("out", ctypes.c_void_p)]


class BatchConfig(ctypes.Structure):
    _fields_ = [("blocks_per_thread_small", ctypes.c_uint32), ("blocks_per_thread_mid", ctypes.c_uint32),
                ("ctas_per_sm", ctypes.c_uint32), ("order", ctypes.c_uint32)]


class ServerConfig(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_batch", ctypes.c_uint32),
                ("fake_executor", ctypes.c_uint32)]


class Completion(ctypes.Structure):
    _fields_ = [("request_id", ctypes.c_uint64), ("channel", ctypes.c_uint32), ("status", ctypes.c_int32),
                ("out_bits", ctypes.c_uint64), ("blocks", ctypes.c_uint64), ("submit_s", ctypes.c_double),
                ("done_s", ctypes.c_double), ("latency_s", ctypes.c_double), ("batched", ctypes.c_uint32),
                ("reserved", ctypes.c_uint32)]


class ServerStats(ctypes.Structure):
    _fields_ = [(k, ctypes.c_uint64) for k in ("submitted", "completed", "rounds", "max_round", "bits_out",
                                               "bytes_in_use", "peak_bytes", "budget_bytes")]


class QextError(RuntimeError):
    def __init__(self, code: int, where: str = ""):
        self.code = code
        super().__init__("%s%s" % (where + ": " if where else "", qext_status_string(code)))


def lib():
    """The loaded libqext (raises if it has not been built)."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise RuntimeError("libqext.so is not built (%s); run __graft_entry__.build()" % LIB_PATH)
    L = ctypes.CDLL(LIB_PATH)
    vp, u32, u64, dbl, i32 = ctypes.c_void_p, ctypes.c_uint32, ctypes.c_uint64, ctypes.c_double, ctypes.c_int
    P = ctypes.POINTER
    L.qext_status_string.argtypes = [i32]
    L.qext_status_string.restype = ctypes.c_char_p
    L.qext_plan_create.argtypes = [u32, u32, dbl, dbl, P(vp)]
    L.qext_destroy.argtypes = [vp]
    L.qext_plan_info.argtypes = [vp, P(u32), P(u32), P(u32), P(dbl), P(u64), P(i32)]
    L.qext_alg1_params.argtypes = [dbl, u32, dbl, dbl, P(u32), P(u32)]
    L.qext_extract.argtypes = [vp, vp, vp, u64, vp, vp]
    L.qext_extract_ex.argtypes = [vp, vp, vp, u64, vp, vp, u32]
    L.qext_pack_samples.argtypes = [u32, vp, u64, vp, vp]
    L.qext_extract_samples.argtypes = [vp, u32, vp, vp, u64, u64, vp, vp]
    L.qext_extract_samples_ex.argtypes = [vp, u32, vp, vp, u64, u64, vp, vp, u32]
    L.qext_device_status.argtypes = [P(i32)]
    L.qext_stream_create.argtypes = [vp, P(vp)]
    L.qext_stream_destroy.argtypes = [vp]
    L.qext_stream_info.argtypes = [vp, P(u64), P(u64), P(u32)]
    L.qext_stream_push.argtypes = [vp, vp, vp, u64, vp, u64, P(u64), vp]
    L.qext_stream_flush.argtypes = [vp, vp, u64, P(u32), vp]
    L.qext_stream_push_samples.argtypes = [vp, u32, vp, vp, u64, vp, u64, P(u64), vp]
    L.qext_stream_state_size.argtypes = [vp]
    L.qext_stream_state_size.restype = ctypes.c_size_t
    L.qext_stream_save.argtypes = [vp, vp, ctypes.c_size_t, P(ctypes.c_size_t), vp]
    L.qext_stream_restore.argtypes = [vp, vp, ctypes.c_size_t, P(vp), vp]
    L.qext_batch_create.argtypes = [vp, u32, P(vp)]
    L.qext_batch_create_samples.argtypes = [vp, u32, P(vp)]
    L.qext_batch_destroy.argtypes = [vp]
    L.qext_batch_get_config.argtypes = [vp, P(BatchConfig), P(u32)]
    L.qext_batch_set_config.argtypes = [vp, P(BatchConfig)]
    L.qext_batch_run.argtypes = [vp, vp]
    L.qext_batch_run_ex.argtypes = [vp, vp, u32]
    L.qext_batch_capture.argtypes = [vp, vp]
    L.qext_batch_launch.argtypes = [vp, vp]
    L.qext_batch_autotune.argtypes = [vp, u32, vp, P(ctypes.c_float)]
    L.qext_batch_run_noalloc.argtypes = [vp, u32, vp]
    L.qext_server_create.argtypes = [P(ServerConfig), P(vp)]
    L.qext_server_destroy.argtypes = [vp]
    L.qext_server_add_channel.argtypes = [vp, vp, P(u32)]
    L.qext_server_submit.argtypes = [vp, u32, u32, vp, vp, u64, vp, u64, P(u64)]
    L.qext_server_poll.argtypes = [vp, P(Completion), u32, P(u32)]
    L.qext_server_drain.argtypes = [vp, dbl]
    L.qext_server_get_stats.argtypes = [vp, P(ServerStats)]
    L.qext_pipeline_create.argtypes = [vp, u32, u64, P(vp)]
    L.qext_pipeline_info.argtypes = [vp, P(u64)]
    L.qext_pipeline_destroy.argtypes = [vp]
    L.qext_pipeline_run.argtypes = [vp, vp, vp, u64, u64, vp]
    L.qext_alg2_plan_create.argtypes = [dbl, u32, u32, u32, u32, P(vp)]
    L.qext_alg2_plan_info.argtypes = [vp, P(u32), P(u32), P(dbl)]
    L.qext_alg2_block_info.argtypes = [vp, u32, P(u32), P(u64), P(u64), P(u64)]
    L.qext_alg2_extract.argtypes = [vp, vp, vp, u32, vp, vp]
    L.qext_alg2_destroy.argtypes = [vp]
    L.qext_sample_histogram.argtypes = [u32, vp, u64, vp, vp]
    L.qext_min_entropy_estimate.argtypes = [u32, P(u64)]
    L.qext_min_entropy_estimate.restype = dbl
    for name in ["qext_plan_create", "qext_destroy", "qext_plan_info", "qext_alg1_params", "qext_extract",
                 "qext_extract_ex", "qext_extract_samples", "qext_extract_samples_ex",
                 "qext_pack_samples", "qext_device_status", "qext_stream_create", "qext_stream_destroy",
                 "qext_stream_info", "qext_stream_push", "qext_stream_push_samples", "qext_stream_flush", "qext_stream_save",
                 "qext_stream_restore", "qext_batch_create", "qext_batch_create_samples", "qext_batch_destroy", "qext_batch_get_config",
                 "qext_batch_set_config", "qext_batch_run", "qext_batch_run_ex", "qext_batch_capture", "qext_batch_launch",
                 "qext_batch_autotune", "qext_batch_run_noalloc", "qext_server_create", "qext_server_destroy",
                 "qext_server_add_channel", "qext_server_submit", "qext_server_poll", "qext_server_drain",
                 "qext_server_get_stats", "qext_pipeline_create", "qext_pipeline_info", "qext_pipeline_destroy",
                 "qext_pipeline_run", "qext_alg2_plan_create", "qext_alg2_plan_info", "qext_alg2_block_info",
                 "qext_alg2_extract", "qext_alg2_destroy", "qext_sample_histogram"]:
        getattr(L, name).restype = i32
    _lib = L
    return L


def _check(rc: int, where: str):
    if rc != QEXT_OK:
        raise QextError(rc, where)


def _ptr(p):
    if p is None:
        return None
    if isinstance(p, int):
        return p
    return int(p.data_ptr())


def _stream(s):
    if s is None:
        import torch
        return int(torch.cuda.current_stream().cuda_stream)
    if isinstance(s, int):
        return s
    return int(s.cuda_stream)


def qext_status_string(code: int) -> str:
    return lib().qext_status_string(code).decode()


class Plan:
    """Owns a qext_plan handle (freed on close / garbage collection)."""

    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().qext_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return qext_plan_info(self)


def qext_plan_create(n: int, m: int, k: float, eps: float) -> Plan:
    h = ctypes.c_void_p()
    _check(lib().qext_plan_create(n, m, k, eps, ctypes.byref(h)), "qext_plan_create")
    return Plan(h.value)


def qext_destroy(plan: Plan) -> None:
    plan.close()


def qext_plan_info(plan: Plan) -> dict:
    q, n_p, m = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_uint32()
    le = ctypes.c_double()
    taps = (ctypes.c_uint64 * 4)()
    sup = ctypes.c_int()
    _check(lib().qext_plan_info(plan.handle, ctypes.byref(q), ctypes.byref(n_p), ctypes.byref(m),
                                ctypes.byref(le), taps, ctypes.byref(sup)), "qext_plan_info")
    return dict(q=q.value, n_p=n_p.value, n=q.value * n_p.value, m=m.value, log2_eps_block=le.value,
                taps=tuple(int(t) for t in taps if t), gpu_supported=int(sup.value))


def qext_alg1_params(N_samples: float, b: int, delta: float, eps: float):
    n_p, q = ctypes.c_uint32(), ctypes.c_uint32()
    _check(lib().qext_alg1_params(N_samples, b, delta, eps, ctypes.byref(n_p), ctypes.byref(q)),
           "qext_alg1_params")
    return n_p.value, q.value


def qext_extract(plan: Plan, x, y, nblocks: int, out, stream=None) -> None:
    _check(lib().qext_extract(plan.handle, _ptr(x), _ptr(y), nblocks, _ptr(out), _stream(stream)),
           "qext_extract")


def qext_extract_ex(plan: Plan, x, y, nblocks: int, out, stream=None, flags: int = 0) -> None:
    _check(lib().qext_extract_ex(plan.handle, _ptr(x), _ptr(y), nblocks, _ptr(out), _stream(stream), flags),
           "qext_extract_ex")


def qext_extract_samples(plan: Plan, b: int, x_samples, y_samples, nsamples: int, nblocks: int, out,
                         stream=None) -> None:
    _check(lib().qext_extract_samples(plan.handle, b, _ptr(x_samples), _ptr(y_samples), nsamples, nblocks,
                                      _ptr(out), _stream(stream)), "qext_extract_samples")


def qext_extract_samples_ex(plan: Plan, b: int, x_samples, y_samples, nsamples: int, nblocks: int, out,
                            stream=None, flags: int = 0) -> None:
    _check(lib().qext_extract_samples_ex(plan.handle, b, _ptr(x_samples), _ptr(y_samples), nsamples, nblocks,
                                         _ptr(out), _stream(stream), flags), "qext_extract_samples_ex")


def qext_pack_samples(b: int, samples, nsamples: int, out, stream=None) -> None:
    _check(lib().qext_pack_samples(b, _ptr(samples), nsamples, _ptr(out), _stream(stream)), "qext_pack_samples")


def qext_device_status() -> int:
    st = ctypes.c_int()
    _check(lib().qext_device_status(ctypes.byref(st)), "qext_device_status")
    return st.value


class Stream:
    """Owns a qext_stream handle (the plan must outlive it)."""

    def __init__(self, handle: int, plan: Plan):
        self.handle = handle
        self.plan = plan

    def close(self):
        if self.handle:
            lib().qext_stream_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qext_stream_create(plan: Plan) -> Stream:
    h = ctypes.c_void_p()
    _check(lib().qext_stream_create(plan.handle, ctypes.byref(h)), "qext_stream_create")
    return Stream(h.value, plan)


def qext_stream_destroy(s: Stream) -> None:
    s.close()


def qext_stream_info(s: Stream):
    a, b, c = ctypes.c_uint64(), ctypes.c_uint64(), ctypes.c_uint32()
    _check(lib().qext_stream_info(s.handle, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), "qext_stream_info")
    return dict(blocks_done=a.value, tail_bits=b.value, pending_bits=c.value)


def qext_stream_push(s: Stream, x, y, nbits: int, out, out_capacity_words: int, stream=None) -> int:
    w = ctypes.c_uint64()
    _check(lib().qext_stream_push(s.handle, _ptr(x), _ptr(y), nbits, _ptr(out), out_capacity_words,
                                  ctypes.byref(w), _stream(stream)), "qext_stream_push")
    return w.value


def qext_stream_push_samples(s: Stream, b: int, x_samples, y_samples, nsamples: int, out, out_capacity_words: int,
                             stream=None) -> int:
    w = ctypes.c_uint64()
    _check(lib().qext_stream_push_samples(s.handle, b, _ptr(x_samples), _ptr(y_samples), nsamples, _ptr(out),
                                          out_capacity_words, ctypes.byref(w), _stream(stream)),
           "qext_stream_push_samples")
    return w.value


def qext_stream_flush(s: Stream, out, out_capacity_words: int, stream=None) -> int:
    b = ctypes.c_uint32()
    _check(lib().qext_stream_flush(s.handle, _ptr(out), out_capacity_words, ctypes.byref(b), _stream(stream)),
           "qext_stream_flush")
    return b.value


def qext_stream_save(s: Stream, stream=None) -> bytes:
    n = lib().qext_stream_state_size(s.handle)
    buf = ctypes.create_string_buffer(n)
    size = ctypes.c_size_t()
    _check(lib().qext_stream_save(s.handle, buf, n, ctypes.byref(size), _stream(stream)), "qext_stream_save")
    return buf.raw[: size.value]


def qext_stream_restore(plan: Plan, state: bytes, stream=None) -> Stream:
    h = ctypes.c_void_p()
    buf = ctypes.create_string_buffer(state, len(state))
    _check(lib().qext_stream_restore(plan.handle, buf, len(state), ctypes.byref(h), _stream(stream)),
           "qext_stream_restore")
    return Stream(h.value, plan)


class Batch:
    """Owns a qext_batch handle; keeps the plans (and buffers) alive."""

    def __init__(self, handle: int, keep):
        self.handle = handle
        self._keep = keep

    def close(self):
        if self.handle:
            lib().qext_batch_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qext_batch_create(items) -> Batch:
    """items: sequence of (plan, x, y, nblocks, out)."""
    arr = (BatchItem * max(1, len(items)))()
    for i, (plan, x, y, nb, out) in enumerate(items):
        arr[i] = BatchItem(plan.handle, _ptr(x), _ptr(y), nb, _ptr(out))
    h = ctypes.c_void_p()
    _check(lib().qext_batch_create(arr, len(items), ctypes.byref(h)), "qext_batch_create")
    return Batch(h.value, [it for it in items])


def qext_batch_create_samples(items) -> Batch:
    """items: sequence of (plan, b, x_samples, y_samples, nsamples, nblocks, out)."""
    arr = (BatchSamplesItem * max(1, len(items)))()
    for i, (plan, b, sx, sy, ns, nb, out) in enumerate(items):
        arr[i] = BatchSamplesItem(plan.handle, b, _ptr(sx), _ptr(sy), ns, nb, _ptr(out))
    h = ctypes.c_void_p()
    _check(lib().qext_batch_create_samples(arr, len(items), ctypes.byref(h)), "qext_batch_create_samples")
    return Batch(h.value, [it for it in items])


def qext_batch_destroy(b: Batch) -> None:
    b.close()


def qext_batch_get_config(b: Batch):
    c = BatchConfig()
    nt = ctypes.c_uint32()
    _check(lib().qext_batch_get_config(b.handle, ctypes.byref(c), ctypes.byref(nt)), "qext_batch_get_config")
    return dict(blocks_per_thread_small=c.blocks_per_thread_small, blocks_per_thread_mid=c.blocks_per_thread_mid,
                ctas_per_sm=c.ctas_per_sm, order=c.order, ntiles=nt.value)


def qext_batch_set_config(b: Batch, blocks_per_thread_small=4, blocks_per_thread_mid=1, ctas_per_sm=3,
                          order=0) -> None:
    c = BatchConfig(blocks_per_thread_small, blocks_per_thread_mid, ctas_per_sm, order)
    _check(lib().qext_batch_set_config(b.handle, ctypes.byref(c)), "qext_batch_set_config")


def qext_batch_run(b: Batch, stream=None) -> None:
    _check(lib().qext_batch_run(b.handle, _stream(stream)), "qext_batch_run")


def qext_batch_run_ex(b: Batch, stream=None, flags: int = 0) -> None:
    _check(lib().qext_batch_run_ex(b.handle, _stream(stream), flags), "qext_batch_run_ex")


def qext_batch_capture(b: Batch, stream=None) -> None:
    _check(lib().qext_batch_capture(b.handle, _stream(stream)), "qext_batch_capture")


def qext_batch_launch(b: Batch, stream=None) -> None:
    _check(lib().qext_batch_launch(b.handle, _stream(stream)), "qext_batch_launch")


def qext_batch_autotune(b: Batch, reps: int = 3, stream=None) -> float:
    ms = ctypes.c_float()
    _check(lib().qext_batch_autotune(b.handle, reps, _stream(stream), ctypes.byref(ms)), "qext_batch_autotune")
    return ms.value


def qext_batch_run_noalloc(items, stream=None) -> None:
    """items: sequence of (plan, x, y, nblocks, out); see include/qext.h."""
    arr = (BatchItem * max(1, len(items)))()
    for i, (plan, x, y, nb, out) in enumerate(items):
        arr[i] = BatchItem(plan.handle, _ptr(x), _ptr(y), nb, _ptr(out))
    _check(lib().qext_batch_run_noalloc(arr, len(items), _stream(stream)), "qext_batch_run_noalloc")


class Server:
    """Owns a qext_server handle; keeps plans and submitted host buffers
    alive until their requests complete."""

    def __init__(self, handle: int):
        self.handle = handle
        self._keep = {}
        self._plans = []

    def close(self):
        if self.handle:
            lib().qext_server_destroy(self.handle)
            self.handle = None
            self._keep.clear()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qext_server_create(hbm_budget_bytes: int, max_batch: int = 256, fake_executor: bool = False) -> Server:
    cfg = ServerConfig(hbm_budget_bytes, max_batch, 1 if fake_executor else 0)
    h = ctypes.c_void_p()
    _check(lib().qext_server_create(ctypes.byref(cfg), ctypes.byref(h)), "qext_server_create")
    return Server(h.value)


def qext_server_destroy(s: Server) -> None:
    s.close()


def qext_server_add_channel(s: Server, plan: Plan) -> int:
    c = ctypes.c_uint32()
    _check(lib().qext_server_add_channel(s.handle, plan.handle, ctypes.byref(c)), "qext_server_add_channel")
    s._plans.append(plan)
    return c.value


def qext_server_submit(s: Server, channel: int, b: int, x_host, y_host, count: int, out_host,
                       out_capacity_words: int) -> int:
    """x_host / y_host / out_host: host tensors (pinned for overlap) or int
    addresses; they are kept alive until the request completes."""
    rid = ctypes.c_uint64()
    _check(lib().qext_server_submit(s.handle, channel, b, _ptr(x_host), _ptr(y_host), count, _ptr(out_host),
                                    out_capacity_words, ctypes.byref(rid)), "qext_server_submit")
    s._keep[rid.value] = (x_host, y_host, out_host)
    return rid.value


def qext_server_poll(s: Server, max_n: int = 1024):
    arr = (Completion * max_n)()
    n = ctypes.c_uint32()
    _check(lib().qext_server_poll(s.handle, arr, max_n, ctypes.byref(n)), "qext_server_poll")
    out = []
    for i in range(n.value):
        c = arr[i]
        out.append(dict(request_id=c.request_id, channel=c.channel, status=c.status, out_bits=c.out_bits,
                        blocks=c.blocks, submit_s=c.submit_s, done_s=c.done_s, latency_s=c.latency_s,
                        batched=bool(c.batched)))
        s._keep.pop(c.request_id, None)
    return out


def qext_server_drain(s: Server, timeout_s: float = 60.0) -> None:
    _check(lib().qext_server_drain(s.handle, timeout_s), "qext_server_drain")


def qext_server_get_stats(s: Server) -> dict:
    st = ServerStats()
    _check(lib().qext_server_get_stats(s.handle, ctypes.byref(st)), "qext_server_get_stats")
    return {k: getattr(st, k) for k, _ in ServerStats._fields_}


class Pipeline:
    def __init__(self, handle: int, plan: Plan):
        self.handle = handle
        self.plan = plan

    def close(self):
        if self.handle:
            lib().qext_pipeline_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def qext_pipeline_create(plan: Plan, b: int, chunk_blocks: int) -> Pipeline:
    h = ctypes.c_void_p()
    _check(lib().qext_pipeline_create(plan.handle, b, chunk_blocks, ctypes.byref(h)), "qext_pipeline_create")
    return Pipeline(h.value, plan)


def qext_pipeline_info(pp: Pipeline) -> dict:
    cb = ctypes.c_uint64()
    _check(lib().qext_pipeline_info(pp.handle, ctypes.byref(cb)), "qext_pipeline_info")
    return dict(chunk_blocks=cb.value)


def qext_pipeline_destroy(pp: Pipeline) -> None:
    pp.close()


def qext_pipeline_run(pp: Pipeline, x_host, y_host, count: int, nblocks: int, out_host) -> None:
    _check(lib().qext_pipeline_run(pp.handle, _ptr(x_host), _ptr(y_host), count, nblocks, _ptr(out_host)),
           "qext_pipeline_run")


class Alg2Plan:
    """Owns a qext_alg2_plan handle (Algorithm 2, growing q_l)."""

    def __init__(self, handle: int):
        self.handle = handle

    def close(self):
        if self.handle:
            lib().qext_alg2_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    @property
    def info(self):
        return qext_alg2_plan_info(self)

    def block(self, l: int) -> dict:
        return qext_alg2_block_info(self, l)


def qext_alg2_plan_create(delta: float, b: int, q1: int, Delta: int, max_blocks: int) -> Alg2Plan:
    h = ctypes.c_void_p()
    _check(lib().qext_alg2_plan_create(delta, b, q1, Delta, max_blocks, ctypes.byref(h)), "qext_alg2_plan_create")
    return Alg2Plan(h.value)


def qext_alg2_plan_info(p: Alg2Plan) -> dict:
    n_p, nb, le = ctypes.c_uint32(), ctypes.c_uint32(), ctypes.c_double()
    _check(lib().qext_alg2_plan_info(p.handle, ctypes.byref(n_p), ctypes.byref(nb), ctypes.byref(le)),
           "qext_alg2_plan_info")
    return dict(n_p=n_p.value, max_blocks=nb.value, log2_error_bound=le.value)


def qext_alg2_block_info(p: Alg2Plan, l: int) -> dict:
    q, ib, ob = ctypes.c_uint32(), ctypes.c_uint64(), ctypes.c_uint64()
    taps = (ctypes.c_uint64 * 4)()
    _check(lib().qext_alg2_block_info(p.handle, l, ctypes.byref(q), ctypes.byref(ib), ctypes.byref(ob), taps),
           "qext_alg2_block_info")
    return dict(q=q.value, in_bit=ib.value, out_bit=ob.value, taps=tuple(int(t) for t in taps if t))


def qext_alg2_extract(p: Alg2Plan, x, y, nblocks: int, out, stream=None) -> None:
    _check(lib().qext_alg2_extract(p.handle, _ptr(x), _ptr(y), nblocks, _ptr(out), _stream(stream)),
           "qext_alg2_extract")


def qext_alg2_destroy(p: Alg2Plan) -> None:
    p.close()


def qext_sample_histogram(b: int, samples, nsamples: int, counts, stream=None) -> None:
    _check(lib().qext_sample_histogram(b, _ptr(samples), nsamples, _ptr(counts), _stream(stream)),
           "qext_sample_histogram")


def qext_min_entropy_estimate(b: int, counts_host) -> float:
    import numpy as np
    c = np.ascontiguousarray(counts_host, dtype=np.uint64)
    return lib().qext_min_entropy_estimate(b, c.ctypes.data_as(ctypes.POINTER(ctypes.c_uint64)))
