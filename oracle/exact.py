"""Brute-force checkers for the N-FHMM oracle (tiny inputs only).

TEST INFRASTRUCTURE: imported only by tests/.  Everything here enumerates;
none of it reuses the recursions of :mod:`oracle.vi`.

* :func:`chain_bruteforce` -- marginals and log normaliser of a single
  chain with emissions exp(phi) by enumerating all N^T paths.
* :func:`product_chain` -- one chain over all N^S joint configurations
  (transition = product of the sources' transitions, emission = sum of the
  sources' phi), solved by path enumeration.
* :func:`log_evidence_exact` -- log P(f) of the Bayesian N-FHMM (Section
  2.2, Eq. 1) for a tiny integer spectrogram: per frame the
  Dirichlet-multinomial mixture over every element assignment of every
  quantum, then all joint state paths.
* :func:`qD_joint_bruteforce` -- the optimal q(D^(1..S)) given q(theta)
  without assuming it factorises over sources: proportional to
  P(D) exp(E_q log P(theta | D)) with the Dirichlet density of Eq. 1
  written out for each joint configuration.
* :func:`elbo_monte_carlo` -- Monte Carlo estimate of E_q[log P] + H[q]
  from samples of q and the model's log density written out term by term.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import digamma, gammaln, logsumexp


def _path_logweights(phi, A, pi):
    T, N = phi.shape
    paths = np.array(list(itertools.product(range(N), repeat=T)), dtype=np.int64)
    with np.errstate(divide="ignore"):
        logA = np.log(A)
        logpi = np.log(pi)
    lw = logpi[paths[:, 0]] + phi[0, paths[:, 0]]
    for t in range(1, T):
        lw = lw + logA[paths[:, t - 1], paths[:, t]] + phi[t, paths[:, t]]
    return paths, lw


def chain_bruteforce(phi, A, pi):
    """All N^T paths of one chain: returns marginals (T, N) and log Z."""
    T, N = phi.shape
    paths, lw = _path_logweights(phi, A, pi)
    logZ = logsumexp(lw)
    p = np.exp(lw - logZ)
    marg = np.zeros((T, N))
    for t in range(T):
        np.add.at(marg[t], paths[:, t], p)
    return marg, float(logZ)


def joint_index(config, N):
    idx = 0
    for n in config:
        idx = idx * N + n
    return idx


def product_chain(phis, As, pis):
    """The S chains as one chain over N^S joint states (Kronecker-product
    transitions, summed phi), solved by enumerating its paths.
    Returns per-source marginals (S, T, N) and log Z of the joint chain."""
    S, T, N = phis.shape
    configs = list(itertools.product(range(N), repeat=S))
    J = len(configs)
    A = np.ones((J, J))
    pi = np.ones(J)
    phi = np.zeros((T, J))
    for a, ca in enumerate(configs):
        pi[a] = np.prod([pis[s][ca[s]] for s in range(S)])
        phi[:, a] = sum(phis[s][:, ca[s]] for s in range(S))
        for b, cb in enumerate(configs):
            A[a, b] = np.prod([As[s][ca[s], cb[s]] for s in range(S)])
    marg_joint, logZ = chain_bruteforce(phi, A, pi)
    marg = np.zeros((S, T, N))
    for a, ca in enumerate(configs):
        for s in range(S):
            marg[s, :, ca[s]] += marg_joint[:, a]
    return marg, logZ


def _block_alpha(config, S, N, K, gamma):
    """alpha(D) of Section 2.2 for one joint configuration."""
    M = S * N * K
    a = np.ones(M)
    for s in range(S):
        k0 = (s * N + config[s]) * K
        a[k0:k0 + K] += gamma
    return a


def frame_loglik_exact(quanta, W, alpha):
    """log P(f_t | alpha) = log sum_{z in [M]^v} prod_v beta_{f_v}(z_v) *
    Gamma(a0)/Gamma(a0 + v) * prod_k Gamma(a_k + n_k)/Gamma(a_k): theta_t
    integrated out of Dir(alpha) times the quanta's categorical draws."""
    M = W.shape[0]
    v = len(quanta)
    if v == 0:
        return 0.0
    a0 = alpha.sum()
    terms = []
    for z in itertools.product(range(M), repeat=v):
        n = np.bincount(np.array(z), minlength=M)
        lt = sum(np.log(W[z[i], quanta[i]]) for i in range(v))
        lt += gammaln(a0) - gammaln(a0 + v) + np.sum(gammaln(alpha + n) - gammaln(alpha))
        terms.append(lt)
    return float(logsumexp(terms))


def log_evidence_exact(V, W, A, pi, S, N, K, gamma):
    """Exact log P(f) of the Bayesian N-FHMM for integer V (T, F) by
    enumerating every joint state path (N^(S T) of them) and, per frame, every
    element assignment of every quantum."""
    T, F = V.shape
    configs = list(itertools.product(range(N), repeat=S))
    J = len(configs)
    frame_ll = np.zeros((T, J))
    for t in range(T):
        quanta = []
        for l in range(F):
            quanta += [l] * int(round(V[t, l]))
        for a, cfg in enumerate(configs):
            frame_ll[t, a] = frame_loglik_exact(quanta, W, _block_alpha(cfg, S, N, K, gamma))
    Aj = np.ones((J, J))
    pij = np.ones(J)
    for a, ca in enumerate(configs):
        pij[a] = np.prod([pi[s][ca[s]] for s in range(S)])
        for b, cb in enumerate(configs):
            Aj[a, b] = np.prod([A[s][ca[s], cb[s]] for s in range(S)])
    _, lw = _path_logweights(frame_ll, Aj, pij)
    return float(logsumexp(lw))


def qD_joint_bruteforce(alpha, A, pi, S, N, K, gamma):
    """q*(D^(1..S)) proportional to P(D) exp(sum_t E_q log Dir(theta_t;
    alpha(D_t))), the joint over all sources' paths (no factorisation
    assumed).  Returns per-source marginals (S, T, N) and the log of its
    normaliser."""
    T, M = alpha.shape
    Elog = digamma(alpha) - digamma(alpha.sum(axis=1, keepdims=True))
    configs = list(itertools.product(range(N), repeat=S))
    J = len(configs)
    phi = np.zeros((T, J))
    for a, cfg in enumerate(configs):
        aD = _block_alpha(cfg, S, N, K, gamma)
        lognorm = gammaln(aD.sum()) - gammaln(aD).sum()
        phi[:, a] = lognorm + Elog @ (aD - 1.0)
    Aj = np.ones((J, J))
    pij = np.ones(J)
    for a, ca in enumerate(configs):
        pij[a] = np.prod([pi[s][ca[s]] for s in range(S)])
        for b, cb in enumerate(configs):
            Aj[a, b] = np.prod([A[s][ca[s], cb[s]] for s in range(S)])
    marg_joint, logZ = chain_bruteforce(phi, Aj, pij)
    marg = np.zeros((S, T, N))
    for a, ca in enumerate(configs):
        for s in range(S):
            marg[s, :, ca[s]] += marg_joint[:, a]
    return marg, logZ


def _dirichlet_logpdf(theta, a):
    return gammaln(a.sum()) - gammaln(a).sum() + np.sum((a - 1.0) * np.log(theta), axis=-1)


def elbo_monte_carlo(V, W, A, pi, alpha, zhat, qD_phi, S, N, K, gamma, n_samples, seed=0):
    """Monte Carlo estimate of E_q[log P(D, theta, Z, f)] - E_q[log q] for
    integer V.  q(theta_t) = Dir(alpha_t); each quantum at frequency l draws
    its element from zhat[t, l]; q(D^(s)) is the chain with emissions
    exp(qD_phi[s]) (paths drawn by enumeration).  Returns (mean, std error)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    T, F = V.shape
    M = W.shape[0]
    quanta = []
    for t in range(T):
        q = []
        for l in range(F):
            q += [l] * int(round(V[t, l]))
        quanta.append(q)
    # q(D^(s)) over whole paths, by enumeration
    path_sets = []
    for s in range(S):
        paths, lw = _path_logweights(qD_phi[s], A[s], pi[s])
        lp = lw - logsumexp(lw)
        path_sets.append((paths, lp))
    with np.errstate(divide="ignore"):
        logA = np.log(A)
        logpi = np.log(pi)
        logW = np.log(W)
        logz = np.log(zhat)
    vals = np.zeros(n_samples)
    for i in range(n_samples):
        lp_joint = 0.0
        lq = 0.0
        D = np.zeros((S, T), dtype=np.int64)
        for s in range(S):
            paths, lp = path_sets[s]
            j = rng.choice(len(paths), p=np.exp(lp))
            D[s] = paths[j]
            lq += lp[j]
            lp_joint += logpi[s, D[s, 0]] + sum(logA[s, D[s, t - 1], D[s, t]] for t in range(1, T))
        for t in range(T):
            theta = rng.dirichlet(alpha[t])
            theta = np.maximum(theta, 1e-300)
            aD = _block_alpha(D[:, t], S, N, K, gamma)
            lp_joint += _dirichlet_logpdf(theta, aD)
            lq += _dirichlet_logpdf(theta, alpha[t])
            for l in quanta[t]:
                z = rng.choice(M, p=zhat[t, l])
                lp_joint += np.log(theta[z]) + logW[z, l]
                lq += logz[t, l, z]
        vals[i] = lp_joint - lq
    return float(vals.mean()), float(vals.std(ddof=1) / np.sqrt(n_samples))
