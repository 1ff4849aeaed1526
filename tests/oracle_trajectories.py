"""Oracle trajectories for the end-to-end validity checks of the GPU tests.

A float32 implementation of the sweep follows the FP64 trajectory closely at
most frames, but at a few near-tie frames (two states with almost equal
surrogate likelihood) rounding differences of 1e-7 relative are amplified
by every sweep, and the trajectories part there while the bound agrees.
Which frames those are is a property of the iteration, not of the
implementation: it is found here by running the FP64 oracle itself with its
state perturbed between sweeps as a float32 implementation's state is --
rounded to float32, and rounded with counts multiplied by (1 + 1e-6 xi),
xi ~ N(0, 1) (five seeds; 1e-6 is the scale of a float32 contraction's
relative error over ~1000 terms).  A frame whose posteriors move by more than a
threshold under any of these perturbations is ill-conditioned at that sweep
(the tests take a tenth of the tolerance: a few random perturbations only
estimate a frame's sensitivity, and the GPU's own rounding is one more,
differently aimed); the GPU's posteriors are held to the tolerance on every
other frame.
"""
import numpy as np

from oracle import vi


def trajectories(p, n_sweeps, noise=1e-6, seeds=(0, 1, 2, 3, 4)):
    """Sweeps 1..n_sweeps of the FP64 oracle from the initial state, and of
    its perturbed runs.  Returns (exact, perturbed): exact[k] = dict(dhat,
    bound, alpha, counts) after sweep k + 1; perturbed[k] = list of d-hat
    arrays after sweep k + 1, one per perturbation."""
    B = vi.element_mask(p.S, p.N, p.K)
    c0, d0 = vi.init_state(p.V, p.W, p.S, p.N, p.K)

    def run(perturb):
        counts, dhat = c0, d0
        out = []
        for _ in range(n_sweeps):
            if perturb is not None:
                counts, dhat = perturb(counts, dhat)
            st = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, counts, dhat, B)
            counts, dhat = st["counts"], st["dhat"]
            out.append(st)
        return out

    def rounding(counts, dhat):
        return (counts.astype(np.float32).astype(np.float64),
                dhat.astype(np.float32).astype(np.float64))

    def noisy(seed):
        rng = np.random.Generator(np.random.PCG64(seed))

        def f(counts, dhat):
            counts, dhat = rounding(counts, dhat)
            return counts * (1.0 + noise * rng.standard_normal(counts.shape)), dhat
        return f

    exact = []
    for st in run(None):
        exact.append(dict(dhat=st["dhat"], alpha=st["alpha"], counts=st["counts"],
                          bound=vi.bound(p.V, p.W, st["alpha"], st["logZ"], p.gamma, p.S,
                                         p.K, Vhat=st["Vhat"])))
    runs = [run(rounding)] + [run(noisy(s)) for s in seeds]
    perturbed = [[r[k]["dhat"] for r in runs] for k in range(n_sweeps)]
    return exact, perturbed


def ill_conditioned(exact_dhat, perturbed_dhats, tol, dilate=2):
    """Boolean mask over frames: frames where any perturbed run's posteriors
    differ from the FP64 ones by more than tol (any source, any state),
    widened by `dilate` frames on each side (the chain couples neighbours)."""
    dev = np.zeros(exact_dhat.shape[1])
    for d in perturbed_dhats:
        dev = np.maximum(dev, np.abs(d - exact_dhat).max(axis=(0, 2)))
    bad = dev > tol
    out = bad.copy()
    for k in range(1, dilate + 1):
        out[k:] |= bad[:-k]
        out[:-k] |= bad[k:]
    return out


def check_sweep_from_own_state(p, counts_in, dhat_in, alpha, counts, dhat, bound, tol_d,
                               tol_rel, tol_bound):
    """One sweep of an implementation, started from its own state
    (counts_in, dhat_in as it held them), against the oracle's sweep from that
    same state: every frame, every output.  Returns the d-hat error."""
    B = vi.element_mask(p.S, p.N, p.K)
    ref = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma,
                   np.asarray(counts_in, np.float64), np.asarray(dhat_in, np.float64), B)
    L_ref = vi.bound(p.V, p.W, ref["alpha"], ref["logZ"], p.gamma, p.S, p.K, Vhat=ref["Vhat"])
    err_d = float(np.max(np.abs(np.asarray(dhat, np.float64) - ref["dhat"])))
    assert err_d <= tol_d, err_d
    a = np.asarray(alpha, np.float64)
    assert np.max(np.abs(a - ref["alpha"]) / ref["alpha"]) <= tol_rel
    c = np.asarray(counts, np.float64)
    big = ref["counts"] > 1e-2 * ref["counts"].max()
    assert np.max(np.abs(c[big] - ref["counts"][big]) / ref["counts"][big]) <= tol_rel
    assert np.max(np.abs(c - ref["counts"])) <= tol_rel * ref["counts"].max()
    assert abs(bound - L_ref) <= tol_bound * abs(L_ref), (bound, L_ref)
    return err_d
