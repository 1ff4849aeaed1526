"""FP64 oracle of exact inference in the original N-FHMM (the comparison
system of Section 5, described at the start of Section 2.2).

TEST INFRASTRUCTURE: imported only by tests/ (and the bench's CPU legs).
It shares no code with the CUDA path.

Model.  Each source s is an N-HMM with N states; state n of source s
selects the K dictionary elements of block (s, n) (element index
k = (s*N + n)*K + j, as everywhere in this repository).  A joint state
c = (d^(1), ..., d^(S)) selects the S*K elements of its S blocks, and frame t
has its own mixture weights theta_t(c) over them: a maximum-likelihood
parameter per (frame, joint state), not a latent variable as in the
Bayesian variant.  Given c, each quantum of frame t picks an element from
theta_t(c) and a frequency from that element's spectrum beta.

One EM iteration, in the order of the algorithm:

* E-step.  For every (t, c) the frame's log-likelihood
  l_t(c) = sum_f V_tf log sum_k theta_t(c)_k beta_k(f); forward-backward on
  the chain over the N^S joint states (transition prod_s A^(s), initial
  prod_s pi^(s), emission exp(l_t(c))) gives the posteriors gamma_t(c) and
  log P(V | theta).
* M-step.  theta_t(c) enters the expected complete-data log-likelihood only
  through the term gamma_t(c) * sum_f V_tf E[log theta_t(c)_z beta_z(f)], so
  its maximiser is the PLCA update
  theta_t(c)_k <- theta_t(c)_k sum_f V_tf beta_k(f) / Vhat_tc(f) / v_t
  whatever the posterior weight (the library's reading where
  gamma_t(c) = 0 leaves it undetermined).

The iteration returns log P(V | theta) of the weights it started from, which
EM cannot decrease from one iteration to the next.  Initial weights:
uniform over each joint state's elements.
"""
from __future__ import annotations

import itertools

import numpy as np
from scipy.special import logsumexp


def joint_states(S: int, N: int) -> np.ndarray:
    """(N^S, S) array of joint states, the last source varying fastest."""
    return np.array(list(itertools.product(range(N), repeat=S)), dtype=np.int64)


def state_elements(S: int, N: int, K: int) -> np.ndarray:
    """(N^S, S*K) element indices selected by each joint state, source by source."""
    cfg = joint_states(S, N)
    out = np.zeros((len(cfg), S * K), dtype=np.int64)
    for c, d in enumerate(cfg):
        out[c] = np.concatenate([(s * N + d[s]) * K + np.arange(K) for s in range(S)])
    return out


def joint_chain(A: np.ndarray, pi: np.ndarray):
    """Transition and initial distribution of the chain over joint states."""
    S = A.shape[0]
    AJ, piJ = A[0], pi[0]
    for s in range(1, S):
        AJ = np.kron(AJ, A[s])
        piJ = np.kron(piJ, pi[s])
    return AJ, piJ


def initial_weights(T: int, S: int, N: int, K: int) -> np.ndarray:
    return np.full((T, N ** S, S * K), 1.0 / (S * K))


def frame_loglik(V: np.ndarray, W: np.ndarray, theta: np.ndarray, elems: np.ndarray):
    """l_t(c) = sum_f V_tf log Vhat_tc(f), Vhat_tc = sum_k theta_t(c)_k beta_k.
    Returns l (T, NC) and Vhat (T, NC, F)."""
    T, NC, _ = theta.shape
    Vhat = np.einsum("tck,ckf->tcf", theta, W[elems])
    with np.errstate(divide="ignore", invalid="ignore"):
        terms = np.where(V[:, None, :] > 0, V[:, None, :] * np.log(Vhat), 0.0)
    return terms.sum(axis=2), Vhat


def forward_backward_joint(l: np.ndarray, AJ: np.ndarray, piJ: np.ndarray):
    """Scaled forward-backward on the joint chain with emissions exp(l):
    posteriors gamma (T, NC) and log P(V | theta)."""
    T, NC = l.shape
    m = l.max(axis=1, keepdims=True)
    e = np.exp(l - m)
    a = np.zeros((T, NC))
    scale = np.zeros(T)
    x = piJ * e[0]
    scale[0] = x.sum()
    a[0] = x / scale[0]
    for t in range(1, T):
        x = (a[t - 1] @ AJ) * e[t]
        scale[t] = x.sum()
        a[t] = x / scale[t]
    b = np.ones(NC)
    gamma = np.zeros((T, NC))
    gamma[T - 1] = a[T - 1]
    for t in range(T - 2, -1, -1):
        b = AJ @ (e[t + 1] * b) / scale[t + 1]
        g = a[t] * b
        gamma[t] = g / g.sum()
    return gamma, float(np.log(scale).sum() + m.sum())


def em_iteration(V, W, A, pi, S, N, K, theta):
    """One EM iteration from weights theta (T, N^S, S*K): returns the new
    weights, log P(V | theta) of the starting weights and the posteriors."""
    elems = state_elements(S, N, K)
    l, Vhat = frame_loglik(V, W, theta, elems)
    AJ, piJ = joint_chain(A, pi)
    gamma, loglik = forward_backward_joint(l, AJ, piJ)
    with np.errstate(divide="ignore", invalid="ignore"):
        Q = np.where(V[:, None, :] > 0, V[:, None, :] / Vhat, 0.0)
    R = np.einsum("tcf,ckf->tck", Q, W[elems])
    new = theta * R
    tot = new.sum(axis=2, keepdims=True)
    new = np.where(tot > 0, new / np.where(tot > 0, tot, 1.0), theta)
    return new, loglik, gamma


def run(V, W, A, pi, S, N, K, n_iter):
    """n_iter iterations from the uniform weights: the log-likelihood before
    each iteration, the final weights and the last posteriors."""
    T = V.shape[0]
    theta = initial_weights(T, S, N, K)
    logliks = []
    gamma = None
    for _ in range(n_iter):
        theta, ll, gamma = em_iteration(V, W, A, pi, S, N, K, theta)
        logliks.append(ll)
    return {"theta": theta, "logliks": np.array(logliks), "gamma": gamma}


def loglik_bruteforce(V, W, A, pi, S, N, K, theta):
    """log P(V | theta) by enumerating every joint state path (tiny T only)."""
    elems = state_elements(S, N, K)
    l, _ = frame_loglik(V, W, theta, elems)
    AJ, piJ = joint_chain(A, pi)
    T, NC = l.shape
    with np.errstate(divide="ignore"):
        lA, lpi = np.log(AJ), np.log(piJ)
    paths = np.array(list(itertools.product(range(NC), repeat=T)), dtype=np.int64)
    lw = lpi[paths[:, 0]] + l[0, paths[:, 0]]
    for t in range(1, T):
        lw = lw + lA[paths[:, t - 1], paths[:, t]] + l[t, paths[:, t]]
    post = np.zeros((T, NC))
    w = np.exp(lw - logsumexp(lw))
    for t in range(T):
        np.add.at(post[t], paths[:, t], w)
    return float(logsumexp(lw)), post
