"""Pins of the exact N-FHMM oracle (the comparison system) against things
other than itself: path enumeration over joint states, the EM guarantee,
the Kronecker structure of the joint chain, and the single-state case that
reduces to per-frame PLCA with its optimality conditions."""
import numpy as np
import pytest

from oracle import nfhmm_exact as ex
from paper_1206_6468_gb300 import synth


def _tiny(S=2, N=2, K=2, F=5, T=4, seed=0):
    p = synth.make_problem(S=S, N=N, K=K, F=F, T=T, self_prob=0.7, energy_sigma=0.5, seed=seed)
    return p


def test_joint_chain_is_the_product_of_the_sources_chains():
    rng = np.random.default_rng(1)
    S, N = 3, 3
    A = rng.dirichlet(np.ones(N), size=(S, N))
    pi = rng.dirichlet(np.ones(N), size=S)
    AJ, piJ = ex.joint_chain(A, pi)
    cfg = ex.joint_states(S, N)
    for c0 in range(len(cfg)):
        assert abs(piJ[c0] - np.prod([pi[s, cfg[c0, s]] for s in range(S)])) < 1e-15
        for c1 in range(len(cfg)):
            want = np.prod([A[s, cfg[c0, s], cfg[c1, s]] for s in range(S)])
            assert abs(AJ[c0, c1] - want) < 1e-15
    assert np.allclose(AJ.sum(axis=1), 1.0)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_forward_backward_matches_path_enumeration(seed):
    p = _tiny(seed=seed)
    rng = np.random.default_rng(seed + 10)
    theta = rng.dirichlet(np.ones(p.S * p.K), size=(p.T, p.N ** p.S))
    elems = ex.state_elements(p.S, p.N, p.K)
    l, _ = ex.frame_loglik(p.V, p.W, theta, elems)
    AJ, piJ = ex.joint_chain(p.A, p.pi)
    gamma, ll = ex.forward_backward_joint(l, AJ, piJ)
    ll_bf, post_bf = ex.loglik_bruteforce(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, theta)
    assert abs(ll - ll_bf) < 1e-10 * max(1.0, abs(ll_bf))
    assert np.max(np.abs(gamma - post_bf)) < 1e-12


def test_em_never_decreases_the_likelihood_and_keeps_weights_normalised():
    p = synth.make_problem(S=2, N=3, K=3, F=17, T=20, self_prob=0.8, energy_sigma=1.0, seed=4)
    r = ex.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, 15)
    ll = r["logliks"]
    assert np.all(np.diff(ll) >= -1e-9 * np.abs(ll[1:]))
    assert ll[-1] > ll[0]
    assert np.allclose(r["theta"].sum(axis=2), 1.0, atol=1e-12)
    assert np.allclose(r["gamma"].sum(axis=1), 1.0, atol=1e-12)


def test_single_joint_state_reduces_to_plca_at_its_optimum():
    """N = 1: one joint state, so the posterior is trivial and each frame's
    weights follow the PLCA (KL-NMF activation) fixed point: at a maximum of
    sum_f V_f log sum_k theta_k beta_k(f) on the simplex, every element in
    use has sum_f V_f beta_k(f) / Vhat(f) = v_t and none exceeds it."""
    p = synth.make_problem(S=2, N=1, K=3, F=11, T=6, self_prob=0.9, energy_sigma=0.0, seed=7)
    r = ex.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, 20000)
    theta = r["theta"][:, 0, :]
    elems = ex.state_elements(p.S, p.N, p.K)[0]
    Vhat = theta @ p.W[elems]
    g = (p.V / Vhat) @ p.W[elems].T          # (T, S*K)
    v = p.V.sum(axis=1, keepdims=True)
    used = theta > 1e-3
    assert np.all(np.abs(g[used] - np.broadcast_to(v, g.shape)[used]) < 1e-5 * np.broadcast_to(v, g.shape)[used])
    assert np.all(g <= v * (1 + 1e-5))
    assert np.allclose(r["gamma"], 1.0)
