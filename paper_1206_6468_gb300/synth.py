"""Seeded synthetic N-FHMM problems (inputs only).

This module samples problems from the generative process of the Bayesian
N-FHMM (Section 2.2): per-source Markov chains over dictionary states, a
spectrum per dictionary element, per-frame mixing weights and Poisson
"quanta" counts.  It holds none of the variational-inference arithmetic
(Eqs. 6-8, forward-backward, the bound); both the CUDA path's tests and
bench and the FP64 oracle's tests draw their inputs from here.

Recipe (the paper's TIMIT workload is not available; these stand in for it,
with its shapes: F = 513 bins from a 1024-point STFT at 16 kHz, two
speakers, N dictionaries of K elements as in Section 5):

* dictionary element k: W[k, :] ~ Dirichlet(0.5 * 1_F), floored at 1e-12
  and renormalised so that it sums to one (beta_l(k) = W[k, l]);
* transitions: self-probability p, the rest (1 - p) / (N - 1) uniformly;
  uniform initial distribution pi;
* states D_t^(s) sampled from each chain;
* weights h_tk ~ Gamma(1, 1) on the K elements of each source's active
  dictionary, 0 elsewhere;
* frame energies e_t = 1 (sigma = 0) or exp(sigma * xi_t), xi_t ~ N(0, 1);
* mean spectrum Vbar_t = e_t * sum_k h_tk W[k, :];
* V = Poisson(1000 * quanta_scale * Vbar) / 1000.

Element index convention: k = (s * N + n) * K + j.
"""
from __future__ import annotations

import dataclasses
from typing import Dict

import numpy as np


@dataclasses.dataclass
class Problem:
    S: int
    N: int
    K: int
    F: int
    T: int
    gamma: float
    V: np.ndarray        # (T, F) float64, frame-contiguous spectrogram
    W: np.ndarray        # (M, F) float64, row k = dictionary element k
    A: np.ndarray        # (S, N, N) float64, A[s, i, j] = P(D_t = j | D_{t-1} = i)
    pi: np.ndarray       # (S, N) float64
    D: np.ndarray        # (S, T) int, the sampled states (ground truth)
    seed: int

    @property
    def M(self) -> int:
        return self.S * self.N * self.K

    def as_f32(self) -> Dict[str, np.ndarray]:
        return {
            "V": np.ascontiguousarray(self.V, dtype=np.float32),
            "W": np.ascontiguousarray(self.W, dtype=np.float32),
            "A": np.ascontiguousarray(self.A, dtype=np.float32),
            "pi": np.ascontiguousarray(self.pi, dtype=np.float32),
        }


def transition_matrix(N: int, self_prob: float) -> np.ndarray:
    if N == 1:
        return np.ones((1, 1))
    A = np.full((N, N), (1.0 - self_prob) / (N - 1))
    np.fill_diagonal(A, self_prob)
    return A


def _sample_frames(rng, W, A, pi, S, N, K, T, energy_sigma, quanta_scale):
    """States, weights, energies and quanta of T frames under model (W, A, pi)."""
    M = S * N * K
    D = np.zeros((S, T), dtype=np.int64)
    for s in range(S):
        if T == 0:
            continue
        D[s, 0] = rng.choice(N, p=pi[s])
        for t in range(1, T):
            D[s, t] = rng.choice(N, p=A[s, D[s, t - 1]])
    h = np.zeros((T, M))
    for s in range(S):
        for t in range(T):
            k0 = (s * N + D[s, t]) * K
            h[t, k0:k0 + K] = rng.gamma(1.0, 1.0, size=K)
    if energy_sigma > 0:
        e = np.exp(energy_sigma * rng.standard_normal(T))
    else:
        e = np.ones(T)
    Vbar = e[:, None] * (h @ W)
    V = rng.poisson(1000.0 * quanta_scale * Vbar) / 1000.0
    return V, D


def _sample_frames_vec(rng, W, A, pi, S, N, K, T, energy_sigma, quanta_scale):
    """The process of _sample_frames with array draws (same distribution,
    different stream): for long spectrograms."""
    M = S * N * K
    D = np.zeros((S, T), dtype=np.int64)
    u = rng.random((S, T))
    for s in range(S):
        if T == 0:
            continue
        cum = np.cumsum(A[s], axis=1)
        cum[:, -1] = 1.0
        D[s, 0] = min(np.searchsorted(np.cumsum(pi[s]), u[s, 0], side="right"), N - 1)
        for t in range(1, T):
            D[s, t] = min(np.searchsorted(cum[D[s, t - 1]], u[s, t], side="right"), N - 1)
    h = np.zeros((T, M))
    rows = np.arange(T)
    for s in range(S):
        g = rng.gamma(1.0, 1.0, size=(T, K))
        k0 = (s * N + D[s]) * K
        for j in range(K):
            h[rows, k0 + j] = g[:, j]
    e = np.exp(energy_sigma * rng.standard_normal(T)) if energy_sigma > 0 else np.ones(T)
    Vbar = e[:, None] * (h @ W)
    V = rng.poisson(1000.0 * quanta_scale * Vbar) / 1000.0
    return V, D


def _sample_model(rng, S, N, K, F, self_prob):
    M = S * N * K
    W = rng.dirichlet(0.5 * np.ones(F), size=M)
    W = np.maximum(W, 1e-12)
    W /= W.sum(axis=1, keepdims=True)
    A = np.stack([transition_matrix(N, self_prob) for _ in range(S)])
    pi = np.full((S, N), 1.0 / N)
    return W, A, pi


def make_problem(S: int, N: int, K: int, F: int, T: int, *, self_prob: float = 0.9,
                 energy_sigma: float = 0.0, quanta_scale: float = 1.0,
                 gamma: float = 1.0, seed: int = 0) -> Problem:
    rng = np.random.Generator(np.random.PCG64(seed))
    W, A, pi = _sample_model(rng, S, N, K, F, self_prob)
    V, D = _sample_frames(rng, W, A, pi, S, N, K, T, energy_sigma, quanta_scale)
    return Problem(S=S, N=N, K=K, F=F, T=T, gamma=gamma, V=V, W=W, A=A, pi=pi,
                   D=D, seed=seed)


@dataclasses.dataclass
class Jobs:
    """Several spectrograms (jobs) drawn from one model."""
    S: int
    N: int
    K: int
    F: int
    gamma: float
    W: np.ndarray
    A: np.ndarray
    pi: np.ndarray
    V: list              # per job (T_j, F) float64
    D: list              # per job (S, T_j) int
    seed: int

    @property
    def lengths(self) -> np.ndarray:
        return np.array([v.shape[0] for v in self.V], dtype=np.int64)

    def problem(self, j: int) -> Problem:
        """Job j as a problem of its own."""
        return Problem(S=self.S, N=self.N, K=self.K, F=self.F, T=self.V[j].shape[0],
                       gamma=self.gamma, V=self.V[j], W=self.W, A=self.A, pi=self.pi,
                       D=self.D[j], seed=self.seed)

    def stacked_V(self) -> np.ndarray:
        """All jobs' frames back to back, float32."""
        return np.ascontiguousarray(np.concatenate(self.V, axis=0), dtype=np.float32)


def make_jobs(S: int, N: int, K: int, F: int, lengths, *, self_prob: float = 0.9,
              energy_sigma: float = 0.0, quanta_scale: float = 1.0, gamma: float = 1.0,
              seed: int = 0) -> Jobs:
    """One model from `seed` and one spectrogram per entry of `lengths`, job j
    drawn from its own stream (seed, j)."""
    rng = np.random.Generator(np.random.PCG64(seed))
    W, A, pi = _sample_model(rng, S, N, K, F, self_prob)
    Vs, Ds = [], []
    for j, T in enumerate(lengths):
        r = np.random.Generator(np.random.PCG64([seed, j]))
        V, D = _sample_frames_vec(r, W, A, pi, S, N, K, int(T), energy_sigma, quanta_scale)
        Vs.append(V)
        Ds.append(D)
    return Jobs(S=S, N=N, K=K, F=F, gamma=gamma, W=W, A=A, pi=pi, V=Vs, D=Ds, seed=seed)


# The workloads, by what they are.
SMALL = dict(S=2, N=4, K=5, F=129, T=200, self_prob=0.9, energy_sigma=0.0)
"""S2 N4 K5 F129 T200, 20 sweeps: sized for the FP64 oracle."""

PAPER_SIZE = dict(S=2, N=40, K=10, F=513, T=3000, self_prob=0.95, energy_sigma=1.5)
"""S2 N40 K10 F513 T3000, 50 sweeps: paper-like size (1024-point STFT)."""

THREE_SOURCE = dict(S=3, N=40, K=10, F=1025, T=6000, self_prob=0.95, energy_sigma=1.5)
"""S3 N40 K10 F1025 T6000: the precision-form workload."""


def batched_lengths(n_jobs: int = 64, lo: int = 500, hi: int = 8000, seed: int = 0) -> np.ndarray:
    """Frame counts of the batched workload: T uniform in [lo, hi]."""
    rng = np.random.Generator(np.random.PCG64(seed + 7919))
    return rng.integers(lo, hi + 1, size=n_jobs)


def small_integer_problem(S: int, N: int, K: int, F: int, T: int, *, max_quanta: int = 3,
                          self_prob: float = 0.7, gamma: float = 1.0, seed: int = 0) -> Problem:
    """Tiny problem with integer quanta counts (v_t <= max_quanta) drawn from
    the generative process itself: states, theta_t ~ Dir(alpha(D_t)), then
    element and frequency per quantum.  For exact-evidence checks."""
    rng = np.random.Generator(np.random.PCG64(seed))
    M = S * N * K
    W = rng.dirichlet(np.ones(F), size=M)
    W = np.maximum(W, 1e-12)
    W /= W.sum(axis=1, keepdims=True)
    A = np.stack([transition_matrix(N, self_prob) for _ in range(S)])
    # make the chains asymmetric so that a transposed A is detectable
    if N > 1:
        for s in range(S):
            A[s] = 0.5 * A[s] + 0.5 * rng.dirichlet(np.ones(N), size=N)
    pi = rng.dirichlet(np.ones(N), size=S)
    D = np.zeros((S, T), dtype=np.int64)
    for s in range(S):
        D[s, 0] = rng.choice(N, p=pi[s])
        for t in range(1, T):
            D[s, t] = rng.choice(N, p=A[s, D[s, t - 1]])
    V = np.zeros((T, F))
    for t in range(T):
        alpha = np.ones(M)
        for s in range(S):
            k0 = (s * N + D[s, t]) * K
            alpha[k0:k0 + K] += gamma
        theta = rng.dirichlet(alpha)
        vt = rng.integers(0, max_quanta + 1)
        for _ in range(vt):
            z = rng.choice(M, p=theta)
            f = rng.choice(F, p=W[z])
            V[t, f] += 1
    return Problem(S=S, N=N, K=K, F=F, T=T, gamma=gamma, V=V, W=W, A=A, pi=pi,
                   D=D, seed=seed)
