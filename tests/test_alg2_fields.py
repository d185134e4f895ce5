"""The fields of Algorithm 2 (Sec. 3.3) up to its 128th block at q_1 = 16,
Delta b = 16: q_l = 16, 32, ..., 2048.  The polynomials P_q of the adopted
rule (the lexicographically first irreducible polynomial of minimum weight,
Sec. 3.2 leaves P open) are stored in tests/golden/alg2_field_polys.txt,
written by make_alg2_field_polys.py with the oracle's search.  They are
pinned here by Berlekamp's criterion on a spread of degrees and by the
oracle's search re-run on two degrees, and the library's plan must use
exactly these polynomials for all 128 fields (its own search, a different
method).  Nothing here touches a GPU."""
import pytest

import oracle
from paper_2402_14607_gb300 import qext
from tests.conftest import read_golden
from tests.test_oracle_pins import irreducible_berlekamp, pdeg


def golden():
    out = {}
    for q, c, b, a in read_golden("alg2_field_polys.txt"):
        out[int(q)] = tuple(int(t) for t in (c, b, a) if int(t))
    return out


def poly_of(q, taps):
    p = (1 << q) | 1
    for t in taps:
        p |= 1 << t
    return p


def test_golden_covers_every_field():
    g = golden()
    assert sorted(g) == list(range(16, 2049, 16))
    for q, taps in g.items():
        assert len(taps) in (1, 3) and all(0 < t < q for t in taps)
        assert list(taps) == sorted(taps, reverse=True)


@pytest.mark.parametrize("q", [16, 400, 1040, 1536, 2048])
def test_golden_polys_irreducible_by_berlekamp(q):
    p = poly_of(q, golden()[q])
    assert pdeg(p) == q
    assert irreducible_berlekamp(p)


@pytest.mark.parametrize("q", [272, 1040])
def test_oracle_search_reproduces_golden(q):
    assert oracle.select_poly(q)[1] == golden()[q]


def test_library_alg2_plan_uses_the_golden_fields():
    p = qext.qext_alg2_plan_create(10.74 / 16, 16, 16, 1, 128)
    g = golden()
    for l in range(128):
        bl = p.block(l)
        assert bl["q"] == 16 * (l + 1)
        assert bl["taps"] == g[bl["q"]], bl
