"""Tile shapes of the tensor-core contractions and their tuner.

Every column tile the tuner may choose is held to the parity tolerances of
the single-job tests (one sweep from the oracle's state: d-hat 1e-5,
alpha-hat and counts 2e-5 relative, bound 1e-6), at the paper's sizes and
at a batch size where each persistent CTA walks several tiles; ring depths
from 2 to the deepest change only the schedule, never the result.  A context
tuned by nfhmm_autotune equals, bit for bit, a context set by hand to the
shape and forward-backward geometry the tuner chose.
"""
import numpy as np
import pytest
from scipy.special import digamma as sp_digamma

from oracle import vi
from paper_1206_6468_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5
BOUND_RTOL = 1e-6
REL_TOL = 2e-5


@pytest.fixture(scope="module")
def nf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def _f32_problem(p):
    for k in ("V", "W", "A", "pi"):
        setattr(p, k, getattr(p, k).astype(np.float32).astype(np.float64))
    return p


@pytest.fixture(scope="module")
def paper_case():
    """The paper-size problem, the oracle's state after two sweeps (float32,
    as a context holds it) and the oracle's next sweep from it."""
    p = _f32_problem(synth.make_problem(seed=3, **synth.PAPER_SIZE))
    B = vi.element_mask(p.S, p.N, p.K)
    counts, dhat = vi.init_state(p.V, p.W, p.S, p.N, p.K)
    for _ in range(2):
        st = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, counts, dhat, B)
        counts, dhat = st["counts"], st["dhat"]
    c32, d32 = counts.astype(np.float32), dhat.astype(np.float32)
    ref = vi.sweep(p.V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, c32.astype(np.float64),
                   d32.astype(np.float64), B)
    ref["bound"] = vi.bound(p.V, p.W, ref["alpha"], ref["logZ"], p.gamma, p.S, p.K,
                            Vhat=ref["Vhat"])
    return p, c32, d32, ref


def _check(p, ref, L, alpha, phi, counts, dhat):
    assert np.max(np.abs(alpha - ref["alpha"]) / ref["alpha"]) <= REL_TOL
    a0 = ref["alpha"].sum(axis=1)
    phi_ref = ref["phi"] + p.gamma * p.K * sp_digamma(a0)[None, :, None]
    assert np.max(np.abs(phi - phi_ref) / (1.0 + np.abs(phi_ref))) <= REL_TOL
    big = ref["counts"] > 1e-2 * ref["counts"].max()
    c = counts.astype(np.float64)
    assert np.max(np.abs(c[big] - ref["counts"][big]) / ref["counts"][big]) <= REL_TOL
    assert np.max(np.abs(c - ref["counts"])) <= REL_TOL * ref["counts"].max()
    assert np.max(np.abs(dhat - ref["dhat"])) <= D_TOL
    assert abs(L - ref["bound"]) <= BOUND_RTOL * abs(ref["bound"])


@pytest.mark.parametrize("gemm1,gemm2,stages,prefetch,epi", [
    (64, 64, 0, 0, 0), (96, 96, 0, 8, 0), (128, 128, 0, 4, 0), (64, 160, 2, 0, 0),
    (96, 160, 3, 16, 0), (128, 96, 2, 0, 0), (128, 128, 0, 0, 1), (64, 96, 3, 4, 1)])
def test_tile_shape_one_sweep_from_oracle_state(nf, paper_case, gemm1, gemm2, stages, prefetch,
                                                epi):
    p, c32, d32, ref = paper_case
    f = p.as_f32()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K, gamma=p.gamma) as ctx:
        ctx.set_tiles(gemm1, gemm2, stages, stages, prefetch, prefetch, epi, epi)
        assert (ctx.tiles()["tile_epi_stage1"], ctx.tiles()["tile_epi_stage2"]) == (epi, epi)
        t = ctx.tiles()
        assert (t["tile_gemm1"], t["tile_gemm2"]) == (gemm1, gemm2)
        if stages:
            assert (t["tile_stages1"], t["tile_stages2"]) == (stages, stages)
        ctx.set_state(c32, d32, 2)
        L = ctx.sweep(1, bound=True)
        alpha = ctx.weights().astype(np.float64)
        phi = ctx.surrogate().astype(np.float64)
        counts, dhat, _ = ctx.get_state()
    _check(p, ref, L, alpha, phi, counts, dhat)


def test_ring_depth_changes_only_the_schedule(nf):
    """The same column tiles with every ring depth give the same state bit for
    bit: the depth orders the copies, not the arithmetic."""
    p = _f32_problem(synth.make_problem(seed=4, **synth.SMALL))
    f = p.as_f32()
    out = []
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K, gamma=p.gamma) as ctx:
        ctx.set_tiles(96, 128)
        deep1, deep2 = ctx.tiles()["tile_stages1"], ctx.tiles()["tile_stages2"]
        for st in range(2, deep1 + 1):
            ctx.set_tiles(stages1=st, stages2=min(st, deep2))
            ctx.reinit(f["V"], f["W"], f["A"], f["pi"])
            L = ctx.sweep(3, bound=True)
            out.append((L, ctx.posteriors(), ctx.get_state()[0]))
    for L, d, c in out[1:]:
        assert L == out[0][0]
        assert np.array_equal(d, out[0][1]) and np.array_equal(c, out[0][2])


def test_bf16_wide_tiles(nf):
    """BF16 contexts also take 192-column tiles; against the FP32 result of
    the same sweep within BF16's tolerance."""
    p = _f32_problem(synth.make_problem(seed=5, **synth.PAPER_SIZE))
    f = p.as_f32()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K, gamma=p.gamma) as a:
        La = a.sweep(2, bound=True)
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K, gamma=p.gamma,
                      precision="bf16") as b:
        b.set_tiles(192, 192)
        assert b.tiles()["tile_gemm1"] == 192
        Lb = b.sweep(2, bound=True)
    assert abs(La - Lb) <= 1e-3 * abs(La)


def test_tile_options_rejected(nf):
    p = synth.make_problem(seed=6, **synth.SMALL)
    f = p.as_f32()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
        for bad in ((160, None), (192, None), (None, 192), (48, None)):
            with pytest.raises(nf.NfhmmError) as e:
                ctx.set_tiles(*bad)
            assert e.value.code == nf.EINVAL
        with pytest.raises(nf.NfhmmError):
            ctx.set_tiles(stages1=1)
        with pytest.raises(nf.NfhmmError):
            ctx.set_tiles(stages1=99)
        assert ctx.tiles()["tile_gemm1"] == 128 and ctx.tiles()["tile_gemm2"] == 160


@pytest.mark.parametrize("job_frames", [None, [1500, 700, 2300, 41, 3000]])
def test_tuned_context_equals_hand_set(nf, job_frames):
    """Autotune (forward-backward form, then tiles), then three sweeps;
    against a context set by hand to the chosen geometry and shape: equal
    bit for bit."""
    if job_frames is None:
        p = _f32_problem(synth.make_problem(seed=7, **synth.PAPER_SIZE))
        V, kw = p.as_f32()["V"], {}
    else:
        jobs = synth.make_jobs(2, 40, 10, 513, job_frames, self_prob=0.95, energy_sigma=1.5,
                               seed=7)
        p = jobs
        V, kw = jobs.stacked_V(), {"job_frames": job_frames}
    W, A, pi = (np.ascontiguousarray(getattr(p, k), dtype=np.float32) for k in ("W", "A", "pi"))
    with nf.VIContext(V, W, A, pi, p.S, p.N, p.K, **kw) as a:
        a.sweep(1)
        tuned = a.autotune(reps=2)
        La = a.sweep(3, bound=True)
        da = a.posteriors()
        ca = a.get_state()[0]
    with nf.VIContext(V, W, A, pi, p.S, p.N, p.K, **kw) as b:
        b.sweep(1)
        b.set_option("fb_chunk", tuned["fb_chunk"])
        b.set_option("fb_group", tuned["fb_group"])
        b.set_option("fb_mode", tuned["fb_mode"])
        t = tuned["tiles"]
        b.set_tiles(t["tile_gemm1"], t["tile_gemm2"], t["tile_stages1"], t["tile_stages2"],
                    t["tile_prefetch1"], t["tile_prefetch2"], t["tile_epi_stage1"],
                    t["tile_epi_stage2"])
        assert b.tiles() == t
        Lb = b.sweep(3, bound=True)
        db = b.posteriors()
        cb = b.get_state()[0]
    print("tuned:", tuned)
    assert La == Lb
    assert np.array_equal(da, db) and np.array_equal(ca, cb)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_staged_epilogue_operand_is_bit_neutral(nf, precision):
    """Staging V and w in shared memory moves the same values by another
    route: the state is bit for bit that of the unstaged epilogue, over a
    batch whose CTAs walk several tiles."""
    lengths = [1500, 700, 2300, 41, 3000]
    jobs = synth.make_jobs(2, 40, 10, 513, lengths, self_prob=0.95, energy_sigma=1.5, seed=9)
    W, A, pi = (np.ascontiguousarray(getattr(jobs, k), dtype=np.float32) for k in ("W", "A", "pi"))
    out = []
    for epi in (0, 1):
        with nf.VIContext(jobs.stacked_V(), W, A, pi, jobs.S, jobs.N, jobs.K,
                          precision=precision, job_frames=lengths) as ctx:
            ctx.set_tiles(128, 128, epi_stage1=epi, epi_stage2=epi)
            L = ctx.sweep(3, bound=True)
            out.append((L, ctx.posteriors(), ctx.get_state()[0]))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1]) and np.array_equal(out[0][2], out[1][2])
