"""Writes table1_oracle_rates.txt: the oracle's convergence rates on the Table 1
workload (section 6: rho = B_{eps,p}(x - a) on [-1,1]^3, eps = 0.4,
a = (1/sqrt(31), 0.2, 0.1), error = max|phi - exact| / max|exact| over the nodes
of [-1,1]^3), fitted over the paper's windows -- 6th order over M = 20..100
(h = 0.1..0.02), 4th order over M = 100..200 (h = 0.02..0.01) -- both on the
paper's own panel counts ("paper") and on the grids the GPU solver uses for
them ("padded": each count padded to the next of 16, 32, 48, 64, 96, 128, 192,
256, the domain extended by whole panels, h unchanged, the error taken at the
nodes of [-1,1]^3).  Calls only oracle/ (and the seeded-input module).

    python tests/golden/make_table1_oracle.py
"""
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

import workloads as w  # noqa: E402
from oracle import closed_form, solve  # noqa: E402

CENTRE = (1 / np.sqrt(31), 0.2, 0.1)
SUPPORTED = (16, 32, 48, 64, 96, 128, 192, 256, 384, 512)
M6 = (20, 28, 40, 56, 80, 100)
M4 = (100, 140, 200)


def padded_problem(M, p):
    """The [-1,1]^3 problem with M panels, embedded in the padded grid (extra
    panels split between the ends, the lower end getting the smaller half)."""
    Mp = min(s for s in SUPPORTED if s >= M)
    lo_extra = (Mp - M) // 2
    h = 2.0 / M
    lo = -1.0 - lo_extra * h
    hi = lo + Mp * h
    return w.scaled_bump((Mp + 1,) * 3, lo=(lo,) * 3, hi=(hi,) * 3, centre=CENTRE, eps=0.4, p=p), lo_extra


def error(M, p, order, padded):
    if padded:
        prob, off = padded_problem(M, p)
    else:
        prob, off = w.scaled_bump((M + 1,) * 3, centre=CENTRE, eps=0.4, p=p), 0
    phi = solve.solve(prob.rho(), prob.h, order, boundary="convolution")
    keep = tuple(slice(off, off + M + 1) for _ in range(3))
    sub = w.scaled_bump((M + 1,) * 3, centre=CENTRE, eps=0.4, p=p)
    ex = closed_form.bump_potential_on_grid(sub)
    return float(np.abs(phi[keep] - ex).max() / np.abs(ex).max())


def rate(Ms, errs):
    return float(np.polyfit(np.log([2.0 / M for M in Ms]), np.log(errs), 1)[0])


def main():
    lines = ["# Oracle convergence rates on the Table 1 workload (section 6), written by",
             "# tests/golden/make_table1_oracle.py (oracle only).  6th order fitted over",
             "# M = 20..100, 4th order over M = 100..200; 'paper' = the paper's panel counts,",
             "# 'padded' = the grids the GPU solver pads them to (error at the nodes of [-1,1]^3).",
             "# columns: differentiability  grids  rate_4th_order  rate_6th_order"]
    for diff, p in ((0, 1), (2, 3), (4, 5), (6, 7), (8, 9)):
        for kind in ("paper", "padded"):
            pad = kind == "padded"
            r6 = rate(M6, [error(M, p, 6, pad) for M in M6])
            r4 = rate(M4, [error(M, p, 4, pad) for M in M4])
            lines.append("%d %s %.3f %.3f" % (diff, kind, r4, r6))
            print(lines[-1], flush=True)
    with open(os.path.join(os.path.dirname(os.path.abspath(__file__)), "table1_oracle_rates.txt"), "w") as f:
        f.write("\n".join(lines) + "\n")


if __name__ == "__main__":
    main()
