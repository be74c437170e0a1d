"""Writes tests/golden/oracle_trajectories.txt.

Calls only ``oracle`` and ``synth``: population after each of the first 64
generations of a few seeded boards, a regression fixture for the oracle.
Run from the repository root: ``python tests/golden/make_golden.py``.
"""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import oracle  # noqa: E402
import synth  # noqa: E402

CASES = [  # (rows, cols, density, seed, torus)
    (64, 64, 0.3, 1, 1),
    (96, 192, 0.5, 2, 1),
    (50, 70, 0.35, 3, 0),
]


def main():
    lines = ["# Population after g = 0..64 generations, computed by the oracle",
             "# (tests/golden/make_golden.py).  Format: rows cols density seed torus: p0 p1 ..."]
    for R, C, p, seed, torus in CASES:
        b = synth.bernoulli_board(R, C, p, seed)
        pops = []
        for g in range(65):
            pops.append(oracle.population(b))
            b = oracle.step(b, torus=bool(torus))
        lines.append("%d %d %g %d %d: %s" % (R, C, p, seed, torus, " ".join(map(str, pops))))
    with open(os.path.join(ROOT, "tests", "golden", "oracle_trajectories.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
