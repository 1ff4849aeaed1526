"""Failure detection on the GPU, without a GPU fault.

* A bounded device wait that gives up.  The test hook
  NFHMM_OPT_TEST_WAIT_TIMEOUT makes the MMA thread of every CTA of the next
  sweep's reconstruction contraction wait 20 ms on an mbarrier that nothing
  completes.  The wait gives up; the CTA winds down -- the TMA producer and
  the epilogue warps see the abort flag and stop waiting, the producer waits
  for its copies in flight and the MMA thread for its MMAs, TMEM is freed --
  and the sweep reports NFHMM_ETIMEOUT through the error word.  The context
  stays usable: restored to the state before the failed sweep, it sweeps on
  bit for bit as a context that never failed.
* Data of probability zero under a chain (an emission that excludes the only
  state the transitions allow): the stateless forward-backward reports it by
  NaN log normalisers, the only output it has.
"""
import time

import numpy as np
import pytest

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


@pytest.mark.parametrize("workload", ["SMALL", "PAPER_SIZE"])
def test_wait_that_gives_up_is_reported_and_context_recovers(nf, workload):
    p = synth.make_problem(seed=21, **getattr(synth, workload))
    f = p.as_f32()

    def ctx():
        return nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K, gamma=p.gamma)

    with ctx() as c:
        c.sweep(2)
        counts, dhat, n = c.get_state()
        c.set_option("test_wait_timeout", 20_000_000)   # 20 ms
        t0 = time.perf_counter()
        with pytest.raises(nf.NfhmmError) as e:
            c.sweep(1, bound=True)
        waited = time.perf_counter() - t0
        assert e.value.code == nf.ETIMEOUT
        assert "wait gave up" in str(e.value)
        # every warp stopped waiting once the MMA thread gave up: far below the
        # 2 s limit of an ordinary wait
        assert waited < 1.5, waited
        c.set_state(counts, dhat, n)
        L = c.sweep(3, bound=True)
        d = c.posteriors()
    with ctx() as r:
        r.sweep(2)
        L_ref = r.sweep(3, bound=True)
        d_ref = r.posteriors()
    assert L == L_ref
    assert np.array_equal(d, d_ref)


def test_wait_hook_rejected_without_tensor_cores(nf):
    p = synth.make_problem(seed=22, **synth.SMALL)
    f = p.as_f32()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K,
                      precision="fp32_simt") as c:
        with pytest.raises(nf.NfhmmError) as e:
            c.set_option("test_wait_timeout", 1000)
        assert e.value.code == nf.EINVAL


def zero_probability_inputs(T=50, N=3):
    """Two chains of N states.  Chain 0 is ordinary.  Chain 1 starts in state
    0 and must move to state 1 (a cyclic permutation), but the emission of
    frame 1 excludes state 1 (phi = -1e4 there: exp underflows to 0), so the
    data have probability zero under chain 1."""
    import torch
    rng = np.random.default_rng(3)
    A = np.stack([0.5 * rng.dirichlet(np.ones(N), size=N) + 0.5 * synth.transition_matrix(N, 0.9),
                  np.roll(np.eye(N), 1, axis=1)])
    pi = np.stack([np.full(N, 1.0 / N), np.eye(N)[0]])
    phi = rng.standard_normal((2, T, N))
    phi[1, 1, 1] = -1e4
    return [torch.tensor(x, dtype=torch.float32).cuda() for x in (phi, A, pi)]


def test_stateless_forward_backward_reports_zero_probability(nf):
    import torch
    phi, A, pi = zero_probability_inputs()
    _, logZ = nf.forward_backward(phi, A, pi)
    torch.cuda.synchronize()
    assert torch.isnan(logZ).all()
    # the next call has its own error word: ordinary inputs give finite results
    _, logZ = nf.forward_backward(phi[:1].contiguous(), A[:1].contiguous(), pi[:1].contiguous())
    torch.cuda.synchronize()
    assert torch.isfinite(logZ).all()
