"""Exact inference in the original N-FHMM (the comparison system) through
the C ABI, against the FP64 oracle oracle/nfhmm_exact.py: the log-likelihood
of every iteration, the joint-state posteriors and the weights."""
import numpy as np
import pytest

from oracle import nfhmm_exact as ex
from paper_1206_6468_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def _problem(S, N, K, F, T, seed):
    p = synth.make_problem(S=S, N=N, K=K, F=F, T=T, self_prob=0.85, energy_sigma=1.0, seed=seed)
    for k in ("V", "W", "A", "pi"):
        setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    return p


@pytest.mark.parametrize("S,N,K,F,T", [(2, 3, 2, 17, 40), (3, 2, 3, 33, 25), (2, 5, 4, 129, 300),
                                       (1, 4, 3, 20, 16)])
def test_exact_em_matches_oracle(nf, S, N, K, F, T):
    p = _problem(S, N, K, F, T, seed=S * 100 + N)
    ref = ex.run(p.V, p.W, p.A, p.pi, S, N, K, 5)
    f = p.as_f32()
    with nf.ExactNFHMM(f["V"], f["W"], f["A"], f["pi"], S, N, K) as x:
        lls = [x.iterate(1) for _ in range(5)]
        gamma = x.posteriors()
        theta = x.weights()
    lls = np.array(lls)
    assert np.all(np.abs(lls - ref["logliks"]) <= 1e-6 * np.abs(ref["logliks"])), (lls, ref["logliks"])
    assert np.all(np.diff(lls) >= -1e-6 * np.abs(lls[1:]))
    assert np.max(np.abs(gamma - ref["gamma"])) <= 1e-4
    big = ref["theta"] > 1e-3
    assert np.max(np.abs(theta[big] - ref["theta"][big]) / ref["theta"][big]) <= 1e-3


def test_exact_em_bf16_close(nf):
    p = _problem(2, 3, 2, 65, 60, seed=9)
    ref = ex.run(p.V, p.W, p.A, p.pi, 2, 3, 2, 3)
    f = p.as_f32()
    with nf.ExactNFHMM(f["V"], f["W"], f["A"], f["pi"], 2, 3, 2, precision="bf16") as x:
        lls = np.array([x.iterate(1) for _ in range(3)])
    assert np.all(np.abs(lls - ref["logliks"]) <= 1e-3 * np.abs(ref["logliks"]))


def test_exact_rejects_bad_sizes(nf):
    p = _problem(2, 3, 2, 17, 10, seed=1)
    f = p.as_f32()
    with pytest.raises(nf.NfhmmError):
        nf.ExactNFHMM(f["V"], f["W"], f["A"], f["pi"], 2, 3, 2, precision="fp32_simt")
