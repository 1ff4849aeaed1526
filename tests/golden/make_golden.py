"""Writes tests/golden/tiny_trajectory.json from the FP64 oracle alone.

The stored values are the oracle's, for a fixed tiny problem (S=2 sources,
N=3 states, K=2 elements, F=7 bins, T=9 frames, generator seed 123, inputs
rounded to float32 as the GPU receives them): the bound after each of four
sweeps from the initial state of Section 3.2's reading (equal weights,
uniform d-hat), and d-hat and alpha-hat after the fourth.  Run from the
repository root:  python tests/golden/make_golden.py
"""
import json
import os
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
sys.path.insert(0, ROOT)

from oracle import vi  # noqa: E402
from paper_1206_6468_gb300 import synth  # noqa: E402

CASE = dict(S=2, N=3, K=2, F=7, T=9, self_prob=0.8, energy_sigma=0.5, seed=123)
SWEEPS = 4


def problem():
    cfg = dict(CASE)
    seed = cfg.pop("seed")
    p = synth.make_problem(seed=seed, **cfg)
    for k in ("V", "W", "A", "pi"):
        setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    return p


def main():
    p = problem()
    ref = vi.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, SWEEPS)
    out = {"case": CASE, "sweeps": SWEEPS, "bounds": [float(x) for x in ref["bounds"]],
           "dhat": np.asarray(ref["dhat"]).tolist(), "alpha": np.asarray(ref["alpha"]).tolist()}
    path = os.path.join(os.path.dirname(os.path.abspath(__file__)), "tiny_trajectory.json")
    with open(path, "w") as f:
        json.dump(out, f, indent=1)
        f.write("\n")


if __name__ == "__main__":
    main()
