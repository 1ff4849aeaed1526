"""Stored fixtures under tests/golden/.

special_values.txt: closed forms of psi and lnGamma (Abramowitz & Stegun
6.3.2, 6.3.3, 6.3.5, 6.1.6) that the oracle's library routines reproduce.
tiny_trajectory.json: written by tests/golden/make_golden.py from the oracle
alone; the oracle must still reproduce it (a change to the oracle's
arithmetic shows here), and the CUDA path is held to it with the FP32
tolerances of the parity tests, without running the oracle.
"""
import json
import os
import sys

import numpy as np
import pytest
from scipy.special import digamma, gammaln

HERE = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")
sys.path.insert(0, HERE)

import make_golden  # noqa: E402


def _trajectory():
    with open(os.path.join(HERE, "tiny_trajectory.json")) as f:
        return json.load(f)


def test_special_values_closed_forms():
    n = 0
    for line in open(os.path.join(HERE, "special_values.txt")):
        if line.startswith("#") or not line.strip():
            continue
        fn, x, v = line.split()
        got = digamma(float(x)) if fn == "digamma" else gammaln(float(x))
        assert abs(got - float(v)) <= 2e-15 * max(1.0, abs(float(v))), (fn, x)
        n += 1
    assert n == 8


def test_oracle_reproduces_stored_trajectory():
    from oracle import vi
    g = _trajectory()
    p = make_golden.problem()
    ref = vi.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, g["sweeps"])
    assert np.allclose(ref["bounds"], g["bounds"], rtol=1e-12, atol=0)
    assert np.allclose(ref["dhat"], g["dhat"], rtol=0, atol=1e-12)
    assert np.allclose(ref["alpha"], g["alpha"], rtol=1e-12, atol=0)


@pytest.mark.gpu
def test_cuda_path_against_stored_trajectory():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    g = _trajectory()
    p = make_golden.problem()
    f = p.as_f32()
    with nfhmm.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K, gamma=p.gamma) as ctx:
        bounds = [ctx.sweep(1, bound=True) for _ in range(g["sweeps"])]
        dhat = ctx.posteriors()
        alpha = ctx.weights()
    assert np.all(np.abs(np.array(bounds) - g["bounds"]) <= 1e-6 * np.abs(g["bounds"]))
    assert np.max(np.abs(dhat - np.array(g["dhat"]))) <= 1e-5
    assert np.max(np.abs(alpha - np.array(g["alpha"])) / np.array(g["alpha"])) <= 2e-5
