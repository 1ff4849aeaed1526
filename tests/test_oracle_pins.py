"""Pins of the FP64 oracle against things other than itself: closed forms,
brute-force enumeration, special cases that reduce to textbook routines,
the exact evidence, a Monte Carlo ELBO and invariants of the update
equations."""
import numpy as np
import pytest
from scipy.special import digamma, gammaln

from oracle import exact, vi
from paper_1206_6468_gb300 import synth

EULER_GAMMA = 0.57721566490153286061


def _rand_chain(rng, N, T, spread=4.0):
    A = rng.dirichlet(np.ones(N), size=N)
    A = 0.6 * A + 0.4 * np.eye(N)          # asymmetric, row-stochastic
    pi = rng.dirichlet(np.ones(N))
    phi = spread * rng.standard_normal((T, N))
    return phi, A, pi


# ---------------------------------------------------------------- digamma etc.

def test_special_functions_closed_forms():
    # psi(1) = -gamma_E, psi(1/2) = -gamma_E - 2 ln 2, psi(n+1) = psi(n) + 1/n
    assert abs(digamma(1.0) + EULER_GAMMA) < 1e-15
    assert abs(digamma(0.5) + EULER_GAMMA + 2 * np.log(2.0)) < 1e-14
    h = 0.0
    for n in range(1, 40):
        assert abs(digamma(n + 1.0) - (-EULER_GAMMA + h + 1.0 / n)) < 1e-13
        h += 1.0 / n
    fact = 1.0
    for n in range(1, 25):
        assert abs(gammaln(n + 1.0) - np.log(fact * n)) < 1e-12 * max(1.0, np.log(fact * n))
        fact *= n


# ------------------------------------------------------------ forward-backward

@pytest.mark.parametrize("N,T,seed", [(1, 5, 0), (2, 7, 1), (3, 6, 2), (3, 1, 3), (2, 2, 4)])
def test_forward_backward_matches_path_enumeration(N, T, seed):
    rng = np.random.default_rng(seed)
    phi, A, pi = _rand_chain(rng, N, T, spread=6.0)
    d, logZ = vi.forward_backward(phi, A, pi)
    d_bf, logZ_bf = exact.chain_bruteforce(phi, A, pi)
    assert np.max(np.abs(d - d_bf)) < 1e-12
    assert abs(logZ - logZ_bf) < 1e-12 * max(1.0, abs(logZ_bf))
    d2, logZ2 = vi.forward_backward_log(phi, A, pi)
    assert np.max(np.abs(d2 - d_bf)) < 1e-12
    assert abs(logZ2 - logZ_bf) < 1e-12 * max(1.0, abs(logZ_bf))


def test_forward_backward_transposed_A_is_detected():
    rng = np.random.default_rng(11)
    phi, A, pi = _rand_chain(rng, 3, 6)
    d_bf, _ = exact.chain_bruteforce(phi, A, pi)
    d_wrong, _ = vi.forward_backward(phi, A.T / A.T.sum(1, keepdims=True), pi)
    assert np.max(np.abs(d_wrong - d_bf)) > 1e-3


def test_forward_backward_pairwise_and_gibbs_identity():
    """log Z = E_q log P(D) + sum_t phi_t(D_t) + H[q] at q = the chain
    posterior, with E_q and H written from the pairwise marginals."""
    rng = np.random.default_rng(5)
    phi, A, pi = _rand_chain(rng, 4, 30, spread=3.0)
    d, logZ, xi = vi.forward_backward(phi, A, pi, want_xi=True)
    assert np.allclose(xi.sum(axis=2), d[:-1], atol=1e-13)
    assert np.allclose(xi.sum(axis=1), d[1:], atol=1e-13)
    Elogp = d[0] @ np.log(pi) + np.sum(xi * np.log(A)[None])
    H = -np.sum(d[0] * np.log(d[0])) - np.sum(xi * np.log(xi / d[:-1, :, None]))
    assert abs(Elogp + np.sum(d * phi) + H - logZ) < 1e-10 * abs(logZ)


def test_long_chain_scaled_matches_log_space():
    rng = np.random.default_rng(6)
    phi, A, pi = _rand_chain(rng, 40, 500, spread=30.0)
    d, logZ = vi.forward_backward(phi, A, pi)
    d2, logZ2 = vi.forward_backward_log(phi, A, pi)
    # log-space sums carry absolute rounding ~ eps * |log Z| (|log Z| ~ 1e4 here)
    assert np.max(np.abs(d - d2)) < 1e-9
    assert abs(logZ - logZ2) < 1e-12 * abs(logZ2)


def test_product_chain_equals_per_source_chains():
    """The N^S joint chain (Kronecker transitions, summed phi) has the
    per-source marginals and log Z = sum_s log Z^(s): q(D) factorises."""
    rng = np.random.default_rng(7)
    S, N, T = 2, 3, 5
    phis = np.zeros((S, T, N))
    As, pis = [], []
    for s in range(S):
        phis[s], A, pi = _rand_chain(rng, N, T)
        As.append(A)
        pis.append(pi)
    marg, logZ = exact.product_chain(phis, As, pis)
    tot = 0.0
    for s in range(S):
        d, lz = vi.forward_backward(phis[s], As[s], pis[s])
        assert np.max(np.abs(d - marg[s])) < 1e-12
        tot += lz
    assert abs(tot - logZ) < 1e-12 * abs(logZ)


# --------------------------------------------------------------- Eqs. 6, 7, 8

def _small_problem(seed=0, **kw):
    args = dict(S=2, N=3, K=2, F=9, T=12, self_prob=0.8, energy_sigma=0.5, quanta_scale=5.0)
    args.update(kw)
    return synth.make_problem(seed=seed, **args)


def test_responsibilities_and_collapsed_counts():
    p = _small_problem(1)
    rng = np.random.default_rng(0)
    alpha = 1.0 + rng.gamma(1.0, 3.0, size=(p.T, p.M))
    for t in range(p.T):
        z = vi.responsibilities(alpha[t], p.W)
        assert np.allclose(z.sum(axis=1), 1.0, atol=1e-14)
    lit = vi.expected_counts_literal(p.V, p.W, alpha)
    col, _ = vi.expected_counts(p.V, p.W, alpha)
    assert np.max(np.abs(lit - col)) < 1e-12 * max(1.0, np.abs(lit).max())
    # every quantum is assigned: sum_k counts_tk = v_t
    assert np.allclose(col.sum(axis=1), p.V.sum(axis=1), rtol=1e-13, atol=1e-13)


def test_initial_counts_are_eq7_at_equal_weights():
    """The initial state's counts (z-hat from equal weights, formed from the
    dictionary's column sums) equal Eq. 7's counts with z-hat materialised
    element by element at any constant alpha-hat, where every psi is equal
    and cancels in the normalisation."""
    p = _small_problem(5)
    counts, _ = vi.init_state(p.V, p.W, p.S, p.N, p.K)
    for a in (1.0, 3.7):
        lit = vi.expected_counts_literal(p.V, p.W, np.full((p.T, p.M), a))
        assert np.max(np.abs(lit - counts)) < 1e-12 * max(1.0, np.abs(lit).max())


def test_dirichlet_update_total_mass():
    """sum_k alpha_tk = v_t + M + gamma S K when each d-hat row sums to 1."""
    p = _small_problem(2)
    B = vi.element_mask(p.S, p.N, p.K)
    counts, dhat = vi.init_state(p.V, p.W, p.S, p.N, p.K)
    for gamma in (0.0, 1.0, 2.5):
        alpha = vi.dirichlet_update(counts, dhat, gamma, B)
        assert np.allclose(alpha.sum(axis=1), p.V.sum(axis=1) + p.M + gamma * p.S * p.K,
                           rtol=1e-13)
        assert alpha.min() >= 1.0


@pytest.mark.parametrize("gamma", [1.0, 0.4, 2.0])
def test_eq8_against_joint_qD_bruteforce(gamma):
    """q*(D) written from the Dirichlet density of Eq. 1 for every joint
    configuration (no factorisation assumed) has the marginals of
    per-source forward-backward on Eq. 8's phi, and log normaliser
    T*lognorm + sum_s log Z^(s)."""
    rng = np.random.default_rng(3)
    S, N, K, T = 2, 2, 3, 4
    M = S * N * K
    alpha = 1.0 + rng.gamma(0.7, 4.0, size=(T, M))
    A = np.stack([_rand_chain(rng, N, 1)[1] for _ in range(S)])
    pi = rng.dirichlet(np.ones(N), size=S)
    B = vi.element_mask(S, N, K)
    phi = vi.surrogate_loglik(alpha, gamma, B)
    marg, logZj = exact.qD_joint_bruteforce(alpha, A, pi, S, N, K, gamma)
    tot = 0.0
    for s in range(S):
        d, lz = vi.forward_backward(phi[s], A[s], pi[s])
        assert np.max(np.abs(d - marg[s])) < 1e-12
        tot += lz
    lognorm = vi.dirichlet_prior_lognorm(M, S, K, gamma)
    assert abs(T * lognorm + tot - logZj) < 1e-11 * max(1.0, abs(logZj))


# ----------------------------------------------------------------- the bound

def _end_of_sweep(p, n_sweeps, gamma=None):
    gamma = p.gamma if gamma is None else gamma
    B = vi.element_mask(p.S, p.N, p.K)
    counts, dhat = vi.init_state(p.V, p.W, p.S, p.N, p.K)
    st = None
    for _ in range(n_sweeps):
        st = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, gamma, counts, dhat, B)
        counts, dhat = st["counts"], st["dhat"]
    return st


def test_bound_collapsed_equals_general():
    p = _small_problem(4, T=6)
    st = _end_of_sweep(p, 3)
    alpha = st["alpha"]
    zhat = np.stack([vi.responsibilities(alpha[t], p.W) for t in range(p.T)])
    xi = []
    for s in range(p.S):
        d, lz, x = vi.forward_backward(st["phi"][s], p.A[s], p.pi[s], want_xi=True)
        xi.append(x)
    Lc = vi.bound(p.V, p.W, alpha, st["logZ"], p.gamma, p.S, p.K, Vhat=st["Vhat"])
    Lg = vi.bound_general(p.V, p.W, p.A, p.pi, alpha, zhat, st["dhat"], xi, p.gamma,
                          p.S, p.N, p.K)
    assert abs(Lc - Lg) < 1e-10 * abs(Lg)


@pytest.mark.parametrize("seed,gamma", [(0, 1.0), (1, 0.5), (2, 3.0)])
def test_bound_monotone(seed, gamma):
    p = _small_problem(seed, T=40, quanta_scale=20.0)
    res = vi.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, gamma, 25)
    L = res["bounds"]
    assert np.all(np.diff(L) >= -1e-12 * np.abs(L[1:]))
    assert L[-1] > L[0]


def test_bound_monotone_small_workload():
    p = synth.make_problem(seed=0, **synth.SMALL)
    res = vi.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, 1.0, 20)
    L = res["bounds"]
    assert np.all(np.diff(L) >= -1e-12 * np.abs(L[1:]))


def _tiny_integer(seed, **kw):
    args = dict(S=2, N=2, K=2, F=4, T=3, max_quanta=3)
    args.update(kw)
    return synth.small_integer_problem(seed=seed, **args)


@pytest.mark.parametrize("seed", [0, 1, 2])
def test_bound_below_exact_evidence(seed):
    """The bound never exceeds the exact log evidence of the Bayesian N-FHMM
    (Dirichlet-multinomial per frame over every element assignment, summed
    over all joint state paths)."""
    p = _tiny_integer(seed)
    logP = exact.log_evidence_exact(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma)
    res = vi.run(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, 15)
    assert np.all(res["bounds"] <= logP + 1e-10)
    assert logP - res["bounds"][-1] < 5.0


def test_exact_evidence_single_element_is_closed_form():
    """S = N = K = 1: theta is a point mass, so log P(f) = sum V log beta."""
    p = _tiny_integer(3, S=1, N=1, K=1, F=3, T=3)
    logP = exact.log_evidence_exact(p.V, p.W, p.A, p.pi, 1, 1, 1, p.gamma)
    assert abs(logP - np.sum(p.V * np.log(p.W[0])[None])) < 1e-12


def test_bound_against_monte_carlo_elbo():
    """The closed-form bound equals a Monte Carlo estimate of
    E_q log P(D, theta, Z, f) - E_q log q with every density written out."""
    p = _tiny_integer(4, T=3)
    st = _end_of_sweep(p, 4)
    alpha = st["alpha"]
    zhat = np.stack([vi.responsibilities(alpha[t], p.W) for t in range(p.T)])
    L = vi.bound(p.V, p.W, alpha, st["logZ"], p.gamma, p.S, p.K, Vhat=st["Vhat"])
    mc, se = exact.elbo_monte_carlo(p.V, p.W, p.A, p.pi, alpha, zhat, st["phi"],
                                    p.S, p.N, p.K, p.gamma, n_samples=6000, seed=1)
    assert abs(mc - L) < 4.5 * se + 1e-3, (mc, se, L)


def test_eq6_is_stationary_for_general_bound():
    """dL/d alpha = 0 at the Eq. 6 update with z-hat and q(D) held fixed
    (central finite differences in random directions)."""
    p = _small_problem(5, T=5, F=6)
    st = _end_of_sweep(p, 2)
    alpha_prev = st["alpha"]
    zhat = np.stack([vi.responsibilities(alpha_prev[t], p.W) for t in range(p.T)])
    xi = [vi.forward_backward(st["phi"][s], p.A[s], p.pi[s], want_xi=True)[2]
          for s in range(p.S)]
    B = vi.element_mask(p.S, p.N, p.K)
    alpha_new = vi.dirichlet_update(st["counts"], st["dhat"], p.gamma, B)

    def L(a):
        return vi.bound_general(p.V, p.W, p.A, p.pi, a, zhat, st["dhat"], xi, p.gamma,
                                p.S, p.N, p.K)

    rng = np.random.default_rng(0)
    h = 1e-4
    for _ in range(4):
        u = rng.standard_normal(alpha_new.shape)
        u /= np.linalg.norm(u)
        g = (L(alpha_new + h * u) - L(alpha_new - h * u)) / (2 * h)
        assert abs(g) < 1e-5, g
    # and it is not stationary at a perturbed point (the check has teeth)
    u = rng.standard_normal(alpha_new.shape)
    a_bad = alpha_new + 0.5 * np.abs(u)
    g_bad = (L(a_bad + h * u) - L(a_bad - h * u)) / (2 * h)
    assert abs(g_bad) > 1e-3


def test_eq7_and_fb_are_maximisers():
    """At fixed alpha, perturbing z-hat (renormalised) or the chain's
    emissions lowers the general bound."""
    p = _small_problem(6, T=5, F=6)
    st = _end_of_sweep(p, 2)
    alpha = st["alpha"]
    zhat = np.stack([vi.responsibilities(alpha[t], p.W) for t in range(p.T)])
    xi = [vi.forward_backward(st["phi"][s], p.A[s], p.pi[s], want_xi=True)[2]
          for s in range(p.S)]
    L0 = vi.bound_general(p.V, p.W, p.A, p.pi, alpha, zhat, st["dhat"], xi, p.gamma,
                          p.S, p.N, p.K)
    rng = np.random.default_rng(1)
    for _ in range(3):
        z2 = zhat * np.exp(0.05 * rng.standard_normal(zhat.shape))
        z2 /= z2.sum(axis=2, keepdims=True)
        assert vi.bound_general(p.V, p.W, p.A, p.pi, alpha, z2, st["dhat"], xi, p.gamma,
                                p.S, p.N, p.K) < L0
        d2 = np.zeros_like(st["dhat"])
        xi2 = []
        for s in range(p.S):
            phi2 = st["phi"][s] + 0.3 * rng.standard_normal(st["phi"][s].shape)
            d2[s], _, x = vi.forward_backward(phi2, p.A[s], p.pi[s], want_xi=True)
            xi2.append(x)
        assert vi.bound_general(p.V, p.W, p.A, p.pi, alpha, zhat, d2, xi2, p.gamma,
                                p.S, p.N, p.K) < L0


# ------------------------------------------------------------- special cases

def test_gamma_zero_gives_prior_marginals():
    p = _small_problem(7, T=15)
    st = _end_of_sweep(p, 3, gamma=0.0)
    assert np.all(st["phi"] == 0.0)
    for s in range(p.S):
        d = p.pi[s].copy()
        for t in range(p.T):
            assert np.allclose(st["dhat"][s, t], d, atol=1e-14)
            d = d @ p.A[s]
        assert abs(st["logZ"][s]) < 1e-12


def test_single_element_model_is_exact():
    """S = N = K = 1: alpha_t = v_t + gamma + 1 and the bound equals the exact
    log evidence sum_lt V_lt log beta_l."""
    p = synth.make_problem(S=1, N=1, K=1, F=7, T=9, self_prob=1.0, quanta_scale=3.0, seed=8)
    for gamma in (1.0, 2.0):
        res = vi.run(p.V, p.W, p.A, p.pi, 1, 1, 1, gamma, 3)
        assert np.allclose(res["alpha"][:, 0], p.V.sum(axis=1) + gamma + 1.0, rtol=1e-14)
        exact_ll = np.sum(p.V * np.log(p.W[0])[None])
        assert np.allclose(res["bounds"], exact_ll, rtol=1e-12)


def _lda_single_document(words, beta, alpha_prior, n_iter, phi0):
    """Textbook LDA variational inference for one document (Blei, Ng &
    Jordan 2003, Sec. 5.2): phi_ni ∝ beta_{i,w_n} exp(psi(gamma_i)),
    gamma_i = alpha_i + sum_n phi_ni; returns gamma and the ELBO (their
    Eq. 15)."""
    phi = phi0.copy()
    g = None
    for _ in range(n_iter):
        g = alpha_prior + phi.sum(axis=0)
        phi = beta[:, words].T * np.exp(digamma(g))[None, :]
        phi /= phi.sum(axis=1, keepdims=True)
    Elog = digamma(g) - digamma(g.sum())
    L = (gammaln(alpha_prior.sum()) - gammaln(alpha_prior).sum()
         + ((alpha_prior - 1) * Elog).sum() + (phi * Elog[None]).sum()
         + (phi * np.log(beta[:, words].T)).sum()
         - gammaln(g.sum()) + gammaln(g).sum() - ((g - 1) * Elog).sum()
         - (phi * np.log(phi)).sum())
    return g, L


def test_single_state_reduces_to_lda():
    """N = 1: d-hat = 1 and each frame is single-document LDA with the
    Dirichlet prior alpha_k = 1 + gamma on every element."""
    p = synth.small_integer_problem(S=2, N=1, K=3, F=5, T=4, max_quanta=6, seed=9)
    gamma = 1.5
    n_sweeps = 6
    res = vi.run(p.V, p.W, p.A, p.pi, p.S, 1, p.K, gamma, n_sweeps)
    assert np.all(res["dhat"] == 1.0)
    Ltot = 0.0
    for t in range(p.T):
        words = np.repeat(np.arange(p.F), p.V[t].astype(int))
        if len(words) == 0:
            phi0 = np.zeros((0, p.M))
        else:
            phi0 = p.W[:, words].T / p.W[:, words].T.sum(axis=1, keepdims=True)
        g, L = _lda_single_document(words, p.W, np.full(p.M, 1.0 + gamma), n_sweeps, phi0)
        assert np.allclose(g, res["alpha"][t], rtol=1e-12)
        Ltot += L
    assert abs(Ltot - res["bounds"][-1]) < 1e-10 * abs(Ltot)


# ---------------------------------------------------------------- separation

def test_separation_invariants():
    p = _small_problem(10, T=20)
    st = _end_of_sweep(p, 3)
    alpha = st["alpha"]
    Vs = vi.separate(p.V, p.W, alpha, p.S, p.N, p.K, masked=False)
    full = (p.V.sum(axis=1)[:, None] * alpha / alpha.sum(axis=1, keepdims=True)) @ p.W
    assert np.allclose(Vs.sum(axis=0), full, rtol=1e-13, atol=1e-15)
    # every dictionary element sums to 1 over frequency (a distribution, Section
    # 2.1), so the mean-weight reconstruction of frame t holds v_t quanta in
    # total, and source s holds its posterior-mean share of them: a wrong
    # scaling of the weights or a wrong element slice per source fails here
    v = p.V.sum(axis=1)
    assert np.allclose(Vs.sum(axis=(0, 2)), v, rtol=1e-12, atol=1e-12)
    NK = p.N * p.K
    for s in range(p.S):
        share = alpha[:, s * NK:(s + 1) * NK].sum(axis=1) / alpha.sum(axis=1)
        assert np.allclose(Vs[s].sum(axis=1), v * share, rtol=1e-12, atol=1e-12)
    Vm = vi.separate(p.V, p.W, alpha, p.S, p.N, p.K, masked=True)
    assert np.allclose(Vm.sum(axis=0), p.V, rtol=1e-13, atol=1e-15)
    assert Vm.min() >= 0.0
    # with the Eq. 7 weights the unmasked sum is the sweep's reconstruction
    Ve = vi.separate(p.V, p.W, alpha, p.S, p.N, p.K, masked=False, weights="expectation")
    assert np.allclose(Ve.sum(axis=0), st["Vhat"], rtol=1e-13)


def test_separation_single_source_is_identity():
    p = _small_problem(11, S=1, T=10)
    st = _end_of_sweep(p, 2)
    Vm = vi.separate(p.V, p.W, st["alpha"], 1, p.N, p.K, masked=True)
    assert np.allclose(Vm[0], p.V, rtol=1e-14, atol=0)
