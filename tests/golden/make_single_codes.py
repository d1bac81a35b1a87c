"""Find, for each single-code workload, the first R draw of its seed that is invertible.

Prints the `skip` values stored in paper_1911_08963_gb300/inputs.py (SINGLE).  Calls only
the CPU oracle (for the rank over F2) and the seeded input generator.

    python tests/golden/make_single_codes.py
"""
import os
import sys

sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__)))))

import oracle as O  # noqa: E402
from paper_1911_08963_gb300 import inputs  # noqa: E402


def first_invertible(n, k, seed, limit=64):
    for skip in range(limit):
        G = inputs.random_code(n, k, seed, skip)
        _, ranks = O.info_sets(G, n, k)
        if ranks == [k, k]:
            return skip
    raise RuntimeError("no invertible draw in %d tries" % limit)


if __name__ == "__main__":
    for name, c in inputs.SINGLE.items():
        print(name, "skip =", first_invertible(c["n"], c["k"], c["seed"]))
