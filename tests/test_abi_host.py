"""Host-side checks of libqext: it loads without a GPU, exports every symbol
declared in include/qext.h, and its plan logic (block factorisation, error
bound, field polynomial) agrees with the oracle.  No GPU work is issued."""
import math
import os
import re

import pytest

import oracle
from paper_2402_14607_gb300 import build as qbuild
from paper_2402_14607_gb300 import qext

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    qbuild.build()
    yield


def declared_functions():
    names = set()
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names |= set(re.findall(r"\b(qext_\w+)\s*\(", text))
    return sorted(names)


def test_library_exports_every_declared_symbol():
    names = declared_functions()
    assert "qext_extract" in names and "qext_plan_create" in names
    L = qext.lib()
    missing = [n for n in names if not hasattr(L, n)]
    assert not missing, missing


def test_status_strings():
    for code in range(-9, 1):
        s = qext.qext_status_string(code)
        assert s.startswith("QEXT_")
    assert "UNKNOWN" in qext.qext_status_string(-1234)


PLAN_CASES = [
    (256, 0, 202, 2.0 ** -9), (1024, 0, 867, 2.0 ** -50), (1024, 0, 867, 2.0 ** -60),
    (4096, 0, 3485, 2.0 ** -52), (4096, 0, 3510, 2.0 ** -52), (1024, 0, 809, 2.0 ** -50),
    (5680, 80, 0.67125 * 5680, 2.0 ** -30), (2048, 40, 1800, 2.0 ** -60), (2048, 0, 1800, 2.0 ** -100),
    (384, 0, 240, 0.5), (512, 7, 450, 2.0 ** -10), (96, 0, 90, 0.25), (2240, 0, 2000, 2.0 ** -70),
]


@pytest.mark.parametrize("n,m,k,eps", PLAN_CASES)
def test_plan_matches_oracle(n, m, k, eps):
    want = oracle.plan(n, m, k, eps)
    p = qext.qext_plan_create(n, m, k, eps)
    got = p.info
    assert (got["n_p"], got["q"], got["m"]) == (want["n_p"], want["q"], want["m"])
    assert abs(got["log2_eps_block"] - want["log2_eps"]) < 1e-9
    assert got["taps"] == want["taps"]
    assert got["gpu_supported"] == (1 if got["q"] in (1, 2, 4, 8, 16, 32, 64) and n % 32 == 0
                                    else 2 if got["q"] == 80 else 0)


@pytest.mark.parametrize("n,m,k,eps,code", [
    (1024, 0, 512, 0.5, qext.QEXT_E_ENTROPY),
    (256, 0, 202, 2.0 ** -40, qext.QEXT_E_PARAM),
    (0, 0, 900, 0.5, qext.QEXT_E_INVAL),           # n = 0
    (1024, 0, 2000, 0.5, qext.QEXT_E_INVAL),       # k > n
    (1024, 0, 900, 1.5, qext.QEXT_E_INVAL),
    (1024, 0, 900, 0.0, qext.QEXT_E_INVAL),
    (1024, 32, 867, 2.0 ** -50, qext.QEXT_E_PARAM),  # m larger than any feasible q
])
def test_plan_rejections(n, m, k, eps, code):
    with pytest.raises(qext.QextError) as e:
        qext.qext_plan_create(n, m, k, eps)
    assert e.value.code == code
    if code != qext.QEXT_E_INVAL:
        with pytest.raises(oracle.PlanError):
            oracle.plan(n, m, k, eps)


@pytest.mark.parametrize("q", [2, 3, 4, 5, 8, 16, 24, 32, 48, 64, 80, 96, 128])
def test_field_polynomial_matches_oracle(q):
    # a plan whose only feasible factorisation has this q: n_p = 32 and a
    # rate close to 1
    n = 32 * q
    p = qext.qext_plan_create(n, 0, n - 0.5, 0.5)
    info = p.info
    if info["q"] != q:
        pytest.skip("plan chose q=%d" % info["q"])
    assert info["taps"] == oracle.select_poly(q)[1]


def test_alg1_params_worked_example():
    assert qext.qext_alg1_params(2.0 ** 51, 16, 10.74 / 16, 2.0 ** -30) == (71, 80)
    assert qext.qext_alg1_params(2.0 ** 51, 16, 10.74 / 16, 2.0 ** -30) == oracle.alg1_params(
        2.0 ** 51, 16, 10.74 / 16, 2.0 ** -30)
    with pytest.raises(qext.QextError) as e:
        qext.qext_alg1_params(1e6, 8, 0.5, 1e-3)
    assert e.value.code == qext.QEXT_E_ENTROPY


def test_paper_q80_plan_has_the_extract_kernels_only():
    p = qext.qext_plan_create(5680, 80, 0.67125 * 5680, 2.0 ** -30)
    info = p.info
    # 2: qext_extract and qext_extract_samples (b = 16) only
    assert (info["n_p"], info["q"], info["gpu_supported"]) == (71, 80, 2)
    assert info["log2_eps_block"] < math.log2(2.0 ** -30)
    # argument checks come before any device work
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract(p, 0, 0, 1, 0, 0)
    assert e.value.code == qext.QEXT_E_INVAL
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract_ex(p, 16, 16, 1, 16, 0, qext.QEXT_F_DIRECT)
    assert e.value.code == qext.QEXT_E_INVAL
    # the other entry points have no q = 80 kernel and refuse the plan
    with pytest.raises(qext.QextError) as e:
        qext.qext_stream_create(p)
    assert e.value.code == qext.QEXT_E_UNSUPPORTED
    with pytest.raises(qext.QextError) as e:
        qext.qext_pipeline_create(p, 16, 1024)
    assert e.value.code == qext.QEXT_E_UNSUPPORTED
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract_samples(p, 12, 16, 16, 10 ** 6, 1, 16, stream=0)
    assert e.value.code == qext.QEXT_E_UNSUPPORTED


def test_extract_argument_checks_without_gpu():
    p = qext.qext_plan_create(1024, 0, 867, 2.0 ** -50)
    for args in [(0, 16, 1, 16), (16, 0, 1, 16), (16, 16, 1, 0), (18, 16, 1, 16), (16, 16, 1, 2)]:
        with pytest.raises(qext.QextError) as e:
            qext.qext_extract(p, *args, stream=0)
        assert e.value.code == qext.QEXT_E_INVAL
    qext.qext_extract(p, 0, 0, 0, 0, stream=0)    # nblocks = 0: nothing to do
    with pytest.raises(qext.QextError) as e:
        qext.qext_pack_samples(17, 16, 4, 16, stream=0)
    assert e.value.code == qext.QEXT_E_INVAL


def test_alg2_plan_checks_without_gpu():
    """Algorithm 2 plans: argument checks before any device work."""
    with pytest.raises(qext.QextError) as e:
        qext.qext_alg2_plan_create(0.5, 16, 16, 1, 4)
    assert e.value.code == qext.QEXT_E_ENTROPY
    with pytest.raises(qext.QextError) as e:
        qext.qext_alg2_plan_create(0.8, 12, 24, 1, 4)     # q_l not multiples of 16
    assert e.value.code == qext.QEXT_E_UNSUPPORTED
    with pytest.raises(qext.QextError) as e:
        qext.qext_alg2_plan_create(0.8, 16, 16, 1, 129)   # q_128 = 2064 > 2048
    assert e.value.code == qext.QEXT_E_UNSUPPORTED
    with pytest.raises(qext.QextError) as e:
        qext.qext_alg2_plan_create(0.8, 16, 0, 1, 4)
    assert e.value.code == qext.QEXT_E_INVAL


def test_samples_argument_checks_without_gpu():
    """qext_extract_samples_ex rejects bad flags, widths, lengths and pointers
    before any device work."""
    p = qext.qext_plan_create(1024, 0, 867, 2.0 ** -50)   # q = 16, n = 1024
    F = qext
    cases = [
        ((12, 16, 16, 1000, 1, 16), 0x100, qext.QEXT_E_INVAL),                                  # unknown flag
        ((12, 16, 16, 1000, 1, 16), F.QEXT_F_TEST_TIMEOUT | F.QEXT_F_WARP_SPECIALIZED, qext.QEXT_E_INVAL),
        ((12, 16, 16, 1000, 1, 16), F.QEXT_F_TEST_TIMEOUT | F.QEXT_F_CTA_TILES, qext.QEXT_E_INVAL),
        ((10, 16, 16, 1000, 1, 16), 0, qext.QEXT_E_UNSUPPORTED),                                # b not 8 / 12 / 16
        ((12, 16, 16, 85, 1, 16), 0, qext.QEXT_E_INVAL),                                         # 85 samples < 1 block
        ((12, 0, 16, 1000, 1, 16), 0, qext.QEXT_E_INVAL),                                        # null x
        ((12, 16, 8, 1000, 1, 16), 0, qext.QEXT_E_INVAL),                                        # y not 16-byte aligned
        ((12, 16, 16, 1000, 1, 2), 0, qext.QEXT_E_INVAL),                                        # out not 4-byte aligned
    ]
    for args, flags, code in cases:
        with pytest.raises(qext.QextError) as e:
            qext.qext_extract_samples_ex(p, *args, stream=0, flags=flags)
        assert e.value.code == code, (args, flags)
    qext.qext_extract_samples_ex(p, 12, 0, 0, 0, 0, 0, stream=0)   # nblocks = 0: nothing to do
    p80 = qext.qext_plan_create(5680, 80, 0.67125 * 5680, 2.0 ** -30)
    with pytest.raises(qext.QextError) as e:
        qext.qext_extract_samples_ex(p80, 16, 16, 16, 10 ** 6, 1, 16, stream=0, flags=qext.QEXT_F_RAW_PREFETCH)
    assert e.value.code == qext.QEXT_E_INVAL    # the q = 80 kernel takes no flags


def test_batch_samples_argument_checks_without_gpu():
    """qext_batch_create_samples checks every item before any device work."""
    p = qext.qext_plan_create(1024, 0, 867, 2.0 ** -50)   # q = 16, n = 1024
    p80 = qext.qext_plan_create(5680, 80, 0.67125 * 5680, 2.0 ** -30)
    cases = [
        ((p, 10, 16, 16, 1000, 1, 16), qext.QEXT_E_UNSUPPORTED),   # b not 8 / 12 / 16
        ((p80, 16, 16, 16, 1000, 1, 16), qext.QEXT_E_UNSUPPORTED),  # q = 80: no batched kernel
        ((p, 12, 16, 16, 85, 1, 16), qext.QEXT_E_INVAL),            # 85 samples < one 1024-bit block
        ((p, 12, 0, 16, 1000, 1, 16), qext.QEXT_E_INVAL),           # null x
        ((p, 12, 16, 8, 1000, 1, 16), qext.QEXT_E_INVAL),           # y not 16-byte aligned
        ((p, 12, 16, 16, 1000, 1, 2), qext.QEXT_E_INVAL),           # out not 4-byte aligned
    ]
    for item, code in cases:
        with pytest.raises(qext.QextError) as e:
            qext.qext_batch_create_samples([item])
        assert e.value.code == code, item


def test_monitor_host_side_without_gpu():
    """The histogram entry checks its arguments before any device work; the
    plug-in min-entropy is host code and agrees with the oracle's."""
    import numpy as np
    for b in (0, 17):
        with pytest.raises(qext.QextError) as e:
            qext.qext_sample_histogram(b, 16, 10, 16, stream=0)
        assert e.value.code == qext.QEXT_E_INVAL
    qext.qext_sample_histogram(12, 0, 0, 0, stream=0)   # no samples: nothing to do
    for samples, counts in [(0, 16), (1, 16), (16, 12)]:  # null / misaligned samples, misaligned counts
        with pytest.raises(qext.QextError) as e:
            qext.qext_sample_histogram(12, samples, 10, counts, stream=0)
        assert e.value.code == qext.QEXT_E_INVAL
    rng = np.random.Generator(np.random.PCG64(5))
    for b in (1, 4, 8, 12, 16):
        counts = rng.integers(0, 1000, 1 << b).astype(np.uint64)
        counts[rng.integers(0, 1 << b)] = 5000
        assert qext.qext_min_entropy_estimate(b, counts) == pytest.approx(oracle.min_entropy_estimate(b, counts),
                                                                           abs=1e-12)
    assert qext.qext_min_entropy_estimate(8, np.zeros(256, np.uint64)) == -1.0     # no samples
    assert qext.qext_min_entropy_estimate(17, np.zeros(1, np.uint64)) == -1.0      # bad width
    flat = np.full(1 << 12, 7, np.uint64)
    assert qext.qext_min_entropy_estimate(12, flat) == pytest.approx(12.0, abs=1e-12)


def test_null_handles_are_rejected_without_gpu():
    """Every entry taking a handle returns QEXT_E_INVAL for a null handle (and
    the destroy entries accept null), with no device work."""
    import ctypes
    L = qext.lib()
    u64, u32 = ctypes.c_uint64(), ctypes.c_uint32()
    INVAL = qext.QEXT_E_INVAL
    calls = [
        (L.qext_plan_info, (None, None, None, None, None, None, None)),
        (L.qext_extract, (None, 16, 16, 1, 16, None)),
        (L.qext_stream_info, (None, None, None, None)),
        (L.qext_stream_push, (None, 16, 16, 32, 16, 1, ctypes.byref(u64), None)),
        (L.qext_stream_flush, (None, 16, 1, ctypes.byref(u32), None)),
        (L.qext_stream_save, (None, 16, 16, None, None)),
        (L.qext_stream_restore, (None, 16, 16, None, None)),
        (L.qext_stream_create, (None, None)),
        (L.qext_batch_get_config, (None, None, None)),
        (L.qext_batch_set_config, (None, None)),
        (L.qext_batch_run, (None, None)),
        (L.qext_batch_capture, (None, None)),
        (L.qext_batch_launch, (None, None)),
        (L.qext_batch_autotune, (None, 1, None, None)),
        (L.qext_batch_create, (None, 1, None)),
        (L.qext_batch_run_noalloc, (None, 1, None)),
        (L.qext_server_add_channel, (None, None, None)),
        (L.qext_server_submit, (None, 0, 12, 16, 16, 1, 16, 1, None)),
        (L.qext_server_poll, (None, None, 0, None)),
        (L.qext_server_drain, (None, 1.0)),
        (L.qext_server_get_stats, (None, None)),
        (L.qext_server_create, (None, None)),
        (L.qext_pipeline_create, (None, 12, 1024, None)),
        (L.qext_pipeline_info, (None, None)),
        (L.qext_pipeline_run, (None, 16, 16, 1, 1, 16)),
        (L.qext_alg2_plan_info, (None, None, None, None)),
        (L.qext_alg2_block_info, (None, 0, None, None, None, None)),
        (L.qext_alg2_extract, (None, 16, 16, 1, 16, None)),
        (L.qext_device_status, (None,)),
    ]
    for fn, args in calls:
        assert fn(*args) == INVAL, fn.__name__
    for fn in (L.qext_destroy, L.qext_stream_destroy, L.qext_batch_destroy, L.qext_server_destroy,
               L.qext_pipeline_destroy, L.qext_alg2_destroy):
        assert fn(None) == qext.QEXT_OK, fn.__name__
    assert L.qext_stream_state_size(None) == 0
