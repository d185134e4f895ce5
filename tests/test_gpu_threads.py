"""Host threads: the first launches of several kernel families, issued at the
same moment from eight threads of a fresh process (cold launch caches), each
on its own CUDA stream, give the same outputs as the same calls made one
after another afterwards."""
import os
import subprocess
import sys
import textwrap

import pytest

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = textwrap.dedent("""
    import sys, threading
    sys.path.insert(0, %r)
    import numpy as np, torch
    from paper_2402_14607_gb300 import qext, workloads
    torch.cuda.init()
    jobs = []
    def words(seed, n):
        return torch.from_numpy(workloads.random_words(seed, n).view(np.int32)).cuda()
    def samples(seed, n, b):
        return torch.from_numpy(workloads.adc_samples(seed, n, b).view(np.int16)).cuda()
    cases = [("q16", 1024, 867, 2.0 ** -50, 5000), ("q64", 4096, 3485, 2.0 ** -52, 700),
             ("q4", 256, 202, 2.0 ** -9, 20000)]
    for name, n, k, eps, nb in cases:
        p = qext.qext_plan_create(n, 0, k, eps)
        x, y = words(len(jobs), nb * n // 32), words(len(jobs) + 100, nb * n // 32)
        out = torch.zeros(nb * p.info["m"] // 32, dtype=torch.int32, device="cuda")
        jobs.append((lambda p=p, x=x, y=y, nb=nb, o=None: (lambda out, st: qext.qext_extract(p, x, y, nb, out, st)), out))
    for name, n, k, eps, b, nb in [("raw16", 1024, 867, 2.0 ** -50, 12, 3000), ("raw4", 256, 202, 2.0 ** -9, 8, 9000),
                                   ("raw64", 4096, 3485, 2.0 ** -52, 12, 400)]:
        p = qext.qext_plan_create(n, 0, k, eps)
        ns = -(-nb * n // b)
        sx, sy = samples(len(jobs), ns, b), samples(len(jobs) + 100, ns, b)
        out = torch.zeros(nb * p.info["m"] // 32, dtype=torch.int32, device="cuda")
        jobs.append((lambda p=p, sx=sx, sy=sy, ns=ns, nb=nb, b=b: (lambda out, st: qext.qext_extract_samples(p, b, sx, sy, ns, nb, out, st)), out))
    p80 = qext.qext_plan_create(5680, 80, 0.67125 * 5680, 2.0 ** -30)
    x80, y80 = words(50, 300 * 5680 // 32 + 1), words(51, 300 * 5680 // 32 + 1)
    o80 = torch.zeros(300 * 80 // 32, dtype=torch.int32, device="cuda")
    jobs.append((lambda: (lambda out, st: qext.qext_extract(p80, x80, y80, 300, out, st)), o80))
    x8, y8 = words(60, 200 * 64 // 32 * 8), words(61, 200 * 64 // 32 * 8)
    p8 = qext.qext_plan_create(512, 0, 400, 0.5)
    o8 = torch.zeros(200 * p8.info["m"] // 32 + 1, dtype=torch.int32, device="cuda")
    jobs.append((lambda: (lambda out, st: qext.qext_extract(p8, x8, y8, 200, out, st)), o8))
    torch.cuda.synchronize()
    start = threading.Barrier(len(jobs))
    errors = []
    def run(i):
        try:
            st = torch.cuda.Stream()
            fn = jobs[i][0]()
            start.wait()
            fn(jobs[i][1], st)
            st.synchronize()
        except Exception as e:  # reported by the parent
            errors.append(repr(e))
    ts = [threading.Thread(target=run, args=(i,)) for i in range(len(jobs))]
    [t.start() for t in ts]
    [t.join() for t in ts]
    if errors:
        print("ERRORS", errors); sys.exit(1)
    torch.cuda.synchronize()
    first = [o.clone() for _, o in jobs]
    for fn, o in jobs:
        o.zero_()
        fn()(o, None)
    torch.cuda.synchronize()
    bad = [i for i, (f, (_, o)) in enumerate(zip(first, jobs)) if not torch.equal(f, o)]
    print("MISMATCH", bad) if bad else print("OK", len(jobs))
    sys.exit(1 if bad else 0)
""") % ROOT


def test_concurrent_first_launches_from_host_threads():
    r = subprocess.run([sys.executable, "-c", CHILD], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0 and "OK 8" in r.stdout, (r.stdout[-2000:], r.stderr[-2000:])
