"""FP64 CPU oracle for variational inference in the Bayesian N-FHMM.

TEST INFRASTRUCTURE.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
``cpu_baseline`` / ``--impl reference`` legs of ``bench.py`` may import or
run anything in this package.  The CUDA library and its binding share no code
with it and never call it.

Every function is plain NumPy/SciPy in float64 and follows the paper
(Mysore & Sahani, "Variational Inference in Non-negative Factorial Hidden
Markov Models for Efficient Audio Source Separation", ICML 2012):

* :mod:`oracle.vi`    -- Eqs. 6, 7, 8, the per-source forward-backward, the
  sweep of Section 3.2, the variational bound, separation (Section 4);
* :mod:`oracle.exact` -- brute-force checkers: path enumeration, the
  product chain over all N^S configurations, the exact evidence of the
  N-FHMM on tiny integer spectrograms, and a Monte Carlo ELBO.

Parity status: every function here is pinned by a ``-m "not gpu"`` test
against something other than itself (closed forms, brute force,
special cases, invariants) except the whole-trajectory values at the
paper-like sizes, which are "parity unpinned" beyond those self-consistency
checks, because the paper prints no intermediate values.
"""

from . import vi, exact  # noqa: F401
