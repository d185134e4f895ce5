"""Writes alg2_field_polys.txt: the field polynomial P_q that the oracle's
search (oracle.select_poly: the lexicographically first irreducible
polynomial of minimum weight) finds for every degree q = 16, 32, ..., 2048,
i.e. every field of Algorithm 2 (Sec. 3.3) with q_1 = 16 and Delta b = 16 up
to its 128th block.  The search at the largest degrees takes minutes, so the
tests read the stored taps and pin them separately (Berlekamp's
irreducibility criterion; the oracle's search re-run on a few degrees).

    python tests/golden/make_alg2_field_polys.py
"""
import os
import sys
import time

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402

OUT = os.path.join(os.path.dirname(os.path.abspath(__file__)), "alg2_field_polys.txt")


def main():
    lines = ["# q c b a : P_q = x^q + x^c + x^b + x^a + 1 (a trinomial x^q + x^c + 1 has b = a = 0)",
             "# written by make_alg2_field_polys.py with the oracle's search (oracle.select_poly)"]
    t0 = time.time()
    for q in range(16, 2048 + 1, 16):
        _, taps = oracle.select_poly(q)
        taps = list(taps) + [0] * (3 - len(taps))
        lines.append("%d %d %d %d" % (q, taps[0], taps[1], taps[2]))
        print(lines[-1], "%.1fs" % (time.time() - t0), flush=True)
    with open(OUT, "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
