"""Variational inference in the Bayesian N-FHMM, plain FP64 (test oracle).

TEST INFRASTRUCTURE: imported only by tests/, __graft_entry__.smoke() and
bench.py's CPU-baseline legs.  Shares no code with the CUDA library.

Notation follows the paper (Section 3.2).  Array layouts:

* ``V``  (T, F): spectrogram, ``V[t, l] = V_lt`` (quanta at frequency l, frame t);
* ``W``  (M, F): dictionary elements, ``W[k, l] = beta_l(k)``, rows sum to 1;
* ``A``  (S, N, N): ``A[s, i, j] = P(D_t^(s) = j | D_{t-1}^(s) = i)`` -- the
  paper's rho^(s) stores the same numbers by columns (Section 2.1);
* ``pi`` (S, N): initial state distributions;
* ``alpha`` (T, M): parameters alpha-hat of q(theta_t);
* ``counts`` (T, M): sum_l V_lt z-hat_tlk, the first term of Eq. 6;
* ``dhat`` (S, T, N): marginals d-hat of q(D^(s));
* ``phi``  (S, T, N): surrogate log-likelihoods phi-hat of Eq. 8.

Element index: k = (s*N + n)*K + j, so the mask B_snk of Section 2.2 is 1
exactly on the K consecutive elements of block (s, n).

Readings where the paper is silent or ambiguous (each is listed in the
design notes):

* Eq. 8 carries the factor gamma.  The paper prints it with gamma = 1
  (Section 2.2 takes gamma = 1); the expectation of log P(theta_t | D_t)
  under q gives gamma * sum_k B_snk <log theta_tk>, and the Dirichlet
  normaliser of alpha(D) does not depend on D because the blocks are
  disjoint and of equal size.
* One sweep is "Eq. 6, then Eqs. 7 and 8 and forward-backward for each
  source" (Section 3.2): alpha-hat is updated from (counts, d-hat), then
  counts (via Eq. 7), phi-hat (Eq. 8) and d-hat (forward-backward) are all
  recomputed from that alpha-hat.  This is coordinate ascent in the two
  blocks {q(theta)} and {q(Z), q(D^(1..S))}.
* Initial state (the paper gives none): d-hat = 1/N (or the prior
  marginals) and z-hat from equal weights, z-hat_tlk = beta_lk / sum_k' beta_lk'.
* Separation (Section 4) uses the posterior-mean weights
  alpha_tk / sum_k alpha_tk scaled by v_t = sum_l V_lt (or, as an option,
  w = exp(psi(alpha)), the weights of Eq. 7); where the mask's denominator
  is zero each source receives V / S.
"""
from __future__ import annotations

import numpy as np
from scipy.special import digamma, gammaln, logsumexp


# --------------------------------------------------------------------- model

def element_mask(S: int, N: int, K: int) -> np.ndarray:
    """B[s, n, k] = 1 iff element k is available when source s is in state n
    (Section 2.2, mask B_snk; disjoint dictionaries of K elements)."""
    M = S * N * K
    B = np.zeros((S, N, M))
    for s in range(S):
        for n in range(N):
            k0 = (s * N + n) * K
            B[s, n, k0:k0 + K] = 1.0
    return B


def prior_alpha(config, gamma: float, B: np.ndarray) -> np.ndarray:
    """alpha_k(D_t) = 1 + gamma * sum_s sum_n delta_tn^(s) B_snk (Section 2.2,
    the Dirichlet parameters of Eq. 1) for one joint configuration."""
    S = B.shape[0]
    a = np.ones(B.shape[2])
    for s in range(S):
        a += gamma * B[s, config[s]]
    return a


# ------------------------------------------------------------ update equations

def dirichlet_update(counts: np.ndarray, dhat: np.ndarray, gamma: float,
                     B: np.ndarray) -> np.ndarray:
    """Eq. 6: alpha_tk = sum_l V_lt z_tlk + gamma sum_s sum_n d_tn^(s) B_snk + 1."""
    return counts + gamma * np.einsum("stn,snk->tk", dhat, B) + 1.0


def responsibilities(alpha_t: np.ndarray, W: np.ndarray) -> np.ndarray:
    """Eq. 7 for one frame, materialised: (F, M) array of z-hat_tlk with
    log z = log beta_l(k) + psi(alpha_tk) - psi(sum_k alpha_tk) - kappa_l,
    kappa_l the log normaliser over k."""
    with np.errstate(divide="ignore"):
        logz = np.log(W.T) + (digamma(alpha_t) - digamma(alpha_t.sum()))[None, :]
    kappa = logsumexp(logz, axis=1, keepdims=True)
    return np.exp(logz - kappa)


def expected_counts_literal(V: np.ndarray, W: np.ndarray, alpha: np.ndarray) -> np.ndarray:
    """sum_l V_lt z-hat_tlk (first term of Eq. 6) with z-hat from Eq. 7
    materialised frame by frame.  Slow; used on small cases."""
    T, M = V.shape[0], W.shape[0]
    out = np.zeros((T, M))
    for t in range(T):
        out[t] = V[t] @ responsibilities(alpha[t], W)
    return out


def expected_counts(V: np.ndarray, W: np.ndarray, alpha: np.ndarray):
    """sum_l V_lt z-hat_tlk without materialising z-hat.

    With w_tk = exp(psi(alpha_tk)), Eq. 7 normalised over k reads
    z-hat_tlk = beta_lk w_tk / Vhat_lt, Vhat_lt = sum_k beta_lk w_tk (the
    psi(sum_k alpha_tk) term and kappa cancel).  Hence
    counts_tk = w_tk * sum_l beta_lk V_lt / Vhat_lt.
    Returns (counts (T, M), Vhat (T, F))."""
    w = np.exp(digamma(alpha))
    Vhat = w @ W
    if np.any((V > 0) & (Vhat <= 0)):
        raise FloatingPointError("Vhat vanishes where V > 0")
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = np.where(V > 0, V / Vhat, 0.0)
    counts = w * (Q @ W.T)
    return counts, Vhat


def surrogate_loglik(alpha: np.ndarray, gamma: float, B: np.ndarray) -> np.ndarray:
    """Eq. 8 (with the factor gamma): phi_tn^(s) =
    gamma * sum_k B_snk (psi(alpha_tk) - psi(sum_k alpha_tk)).  (S, T, N)."""
    E = digamma(alpha) - digamma(alpha.sum(axis=1, keepdims=True))
    return gamma * np.einsum("snk,tk->stn", B, E)


# ----------------------------------------------------------- forward-backward

def forward_backward(phi: np.ndarray, A: np.ndarray, pi: np.ndarray, want_xi: bool = False):
    """Marginals of q(D) proportional to pi(D_1) prod_t A(D_{t-1}, D_t)
    prod_t exp(phi_t(D_t)) -- the q(D^(s)) of Section 3.2, found by the
    forward-backward algorithm (Rabiner 1989) in scaled form.

    phi (T, N), A (N, N) row-stochastic, pi (N,).  Emissions are
    exp(phi_t - max_n phi_t); log Z adds the maxima back.
    Returns dhat (T, N), log Z (float) and, if asked, the pairwise marginals
    xi[t-1, i, j] = q(D_{t-1} = i, D_t = j), t = 1..T-1."""
    T, N = phi.shape
    m = phi.max(axis=1)
    e = np.exp(phi - m[:, None])
    a = np.zeros((T, N))
    c = np.zeros(T)
    x = pi * e[0]
    c[0] = x.sum()
    a[0] = x / c[0]
    for t in range(1, T):
        x = e[t] * (a[t - 1] @ A)
        c[t] = x.sum()
        a[t] = x / c[t]
    b = np.ones((T, N))
    for t in range(T - 1, 0, -1):
        b[t - 1] = (A @ (e[t] * b[t])) / c[t]
    dhat = a * b
    dhat /= dhat.sum(axis=1, keepdims=True)
    logZ = float(np.log(c).sum() + m.sum())
    if not want_xi:
        return dhat, logZ
    xi = np.zeros((max(T - 1, 0), N, N))
    for t in range(1, T):
        xi[t - 1] = a[t - 1][:, None] * A * (e[t] * b[t])[None, :] / c[t]
    return dhat, logZ, xi


def forward_backward_log(phi: np.ndarray, A: np.ndarray, pi: np.ndarray):
    """The same marginals and log Z computed in log space (no scaling)."""
    T, N = phi.shape
    with np.errstate(divide="ignore"):
        logA = np.log(A)
        logpi = np.log(pi)
    la = np.zeros((T, N))
    la[0] = logpi + phi[0]
    for t in range(1, T):
        la[t] = phi[t] + logsumexp(la[t - 1][:, None] + logA, axis=0)
    lb = np.zeros((T, N))
    for t in range(T - 1, 0, -1):
        lb[t - 1] = logsumexp(logA + (phi[t] + lb[t])[None, :], axis=1)
    logZ = float(logsumexp(la[T - 1]))
    dhat = np.exp(la + lb - logZ)
    return dhat, logZ


# --------------------------------------------------------------------- sweep

def init_state(V: np.ndarray, W: np.ndarray, S: int, N: int, K: int,
               A: np.ndarray | None = None, pi: np.ndarray | None = None,
               mode: int = 0):
    """Initial (counts, dhat).  z-hat from equal weights (every psi equal in
    Eq. 7): z-hat_tlk = beta_lk / sum_k' beta_lk'.  dhat = 1/N (mode 0) or the
    prior marginals pi A^(t) (mode 1)."""
    T = V.shape[0]
    colsum = W.sum(axis=0)                      # sum_k beta_lk, (F,)
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = np.where(V > 0, V / colsum[None, :], 0.0)
    counts = Q @ W.T
    if mode == 0:
        dhat = np.full((S, T, N), 1.0 / N)
    else:
        dhat = np.zeros((S, T, N))
        for s in range(S):
            d = pi[s].copy()
            for t in range(T):
                dhat[s, t] = d
                d = d @ A[s]
    return counts, dhat


def sweep(V, W, A, pi, S, N, K, gamma, counts, dhat, B=None):
    """One sweep of Section 3.2: Eq. 6, then Eq. 7 (into the counts of
    Eq. 6), Eq. 8 and forward-backward for each source, all from the new
    alpha-hat."""
    if B is None:
        B = element_mask(S, N, K)
    alpha = dirichlet_update(counts, dhat, gamma, B)
    new_counts, Vhat = expected_counts(V, W, alpha)
    phi = surrogate_loglik(alpha, gamma, B)
    new_dhat = np.zeros_like(dhat)
    logZ = np.zeros(S)
    for s in range(S):
        new_dhat[s], logZ[s] = forward_backward(phi[s], A[s], pi[s])
    return {"alpha": alpha, "counts": new_counts, "dhat": new_dhat, "phi": phi,
            "logZ": logZ, "Vhat": Vhat}


def run(V, W, A, pi, S, N, K, gamma, n_sweeps, init_mode=0, with_bound=True):
    """n sweeps from the initial state; returns the last sweep's state and
    the bound after each sweep."""
    B = element_mask(S, N, K)
    counts, dhat = init_state(V, W, S, N, K, A, pi, init_mode)
    bounds = []
    st = None
    for _ in range(n_sweeps):
        st = sweep(V, W, A, pi, S, N, K, gamma, counts, dhat, B)
        counts, dhat = st["counts"], st["dhat"]
        if with_bound:
            bounds.append(bound(V, W, st["alpha"], st["logZ"], gamma, S, K, Vhat=st["Vhat"]))
    if st is None:
        st = {"counts": counts, "dhat": dhat}
    st["bounds"] = np.array(bounds)
    return st


# --------------------------------------------------------------------- bound

def dirichlet_prior_lognorm(M: int, S: int, K: int, gamma: float) -> float:
    """log Gamma(sum_k alpha_k(D)) - sum_k log Gamma(alpha_k(D)) for the
    Dirichlet of Eq. 1: the same for every D because the blocks are disjoint
    and all of size K."""
    return float(gammaln(M + gamma * S * K) - S * K * gammaln(1.0 + gamma))


def bound(V, W, alpha, logZ, gamma, S, K, Vhat=None):
    """Variational lower bound at a state (alpha, z*(alpha), d*(alpha)) that
    ends a sweep: z-hat from Eq. 7 and d-hat from forward-backward on the
    phi-hat of Eq. 8, both for this alpha.  ``logZ`` are the per-source
    forward-backward log normalisers for phi-hat of Eq. 8.

    L = sum_t [ sum_l V_lt log Vhat_lt - v_t psi(alpha_t0)
              + log G(M + gamma S K) - S K log G(1 + gamma)
              - log G(alpha_t0) + sum_k log G(alpha_tk)
              - sum_k (alpha_tk - 1)(psi(alpha_tk) - psi(alpha_t0)) ]
        + sum_s log Z^(s)
    (the paper prints no bound; this follows from Eq. 1 and the factorised
    posterior of Section 3.2, and equals :func:`bound_general` there)."""
    M = alpha.shape[1]
    a0 = alpha.sum(axis=1)
    psi0 = digamma(a0)
    E = digamma(alpha) - psi0[:, None]
    if Vhat is None:
        Vhat = np.exp(digamma(alpha)) @ W
    v = V.sum(axis=1)
    with np.errstate(divide="ignore", invalid="ignore"):
        VlogVhat = np.where(V > 0, V * np.log(Vhat), 0.0).sum(axis=1)
    const = dirichlet_prior_lognorm(M, S, K, gamma)
    per_t = (VlogVhat - v * psi0 + const - gammaln(a0) + gammaln(alpha).sum(axis=1)
             - ((alpha - 1.0) * E).sum(axis=1))
    return float(per_t.sum() + np.sum(logZ))


def _xlogy(x, y):
    with np.errstate(divide="ignore", invalid="ignore"):
        return np.where(x > 0, x * np.log(np.where(x > 0, y, 1.0)), 0.0)


def bound_general(V, W, A, pi, alpha, zhat, dhat, xi, gamma, S, N, K):
    """The bound written term by term for any q in the factorised family:
    q(theta_t) = Dir(alpha_t), q(Z_tv) = z-hat_{t, f_tv, .} (``zhat`` (T, F, M)),
    q(D^(s)) a Markov chain with marginals ``dhat[s]`` and pairwise marginals
    ``xi[s]`` ((T-1, N, N)).

    L = E_q log P(D, theta, Z, f) + H[q], with
    E log P(theta_t | D_t) = lognorm + sum_k (E_q alpha_k(D_t) - 1) <log theta_tk>,
    E log P(Z, f | theta) = sum_l V_lt sum_k z_tlk (<log theta_tk> + log beta_lk)."""
    T, M = alpha.shape
    B = element_mask(S, N, K)
    a0 = alpha.sum(axis=1)
    E = digamma(alpha) - digamma(a0)[:, None]
    # Dirichlet prior of Eq. 1, its normaliser evaluated at one configuration
    aD = prior_alpha([0] * S, gamma, B)
    lognorm = gammaln(aD.sum()) - gammaln(aD).sum()
    Eam1 = gamma * np.einsum("stn,snk->tk", dhat, B)
    L_theta_prior = T * lognorm + (Eam1 * E).sum()
    # quanta: elements and frequencies
    with np.errstate(divide="ignore"):
        logW = np.log(W.T)                               # (F, M)
    L_zf = np.einsum("tl,tlk->", V, zhat * (E[:, None, :] + logW[None]))
    H_z = -np.einsum("tl,tlk->", V, _xlogy(zhat, zhat))
    H_theta = (-gammaln(a0) + gammaln(alpha).sum(axis=1) - ((alpha - 1.0) * E).sum(axis=1)).sum()
    L_D = 0.0
    for s in range(S):
        with np.errstate(divide="ignore"):
            logA = np.log(A[s])
            logpi = np.log(pi[s])
        ElogpD = float(np.sum(np.where(dhat[s, 0] > 0, dhat[s, 0] * logpi, 0.0)))
        ElogpD += float(np.sum(np.where(xi[s] > 0, xi[s] * logA[None], 0.0)))
        HqD = -float(np.sum(_xlogy(dhat[s, 0], dhat[s, 0])))
        if T > 1:
            cond = xi[s] / np.maximum(dhat[s, :-1, :, None], 1e-300)
            HqD -= float(np.sum(_xlogy(xi[s], cond)))
        L_D += ElogpD + HqD
    return float(L_theta_prior + L_zf + H_z + H_theta + L_D)


# --------------------------------------------------------------- separation

def separate(V, W, alpha, S, N, K, masked=True, weights="mean"):
    """Section 4: Vhat^(s)_lt, a combination of source s's dictionary
    elements weighted by the estimated mixture weights; with ``masked`` the
    refinement V*^(s)_lt = V_lt Vhat^(s)_lt / sum_s' Vhat^(s')_lt.
    weights = "mean": v_t * alpha_tk / sum_k alpha_tk; "expectation":
    exp(psi(alpha_tk)).  Returns (S, T, F)."""
    T, F = V.shape
    if weights == "mean":
        wts = V.sum(axis=1)[:, None] * alpha / alpha.sum(axis=1, keepdims=True)
    else:
        wts = np.exp(digamma(alpha))
    out = np.zeros((S, T, F))
    for s in range(S):
        ks = slice(s * N * K, (s + 1) * N * K)
        out[s] = wts[:, ks] @ W[ks]
    if masked:
        den = out.sum(axis=0)
        with np.errstate(divide="ignore", invalid="ignore"):
            out = np.where(den[None] > 0, V[None] * out / den[None], V[None] / S)
    return out
