"""Batches of jobs sharing one model, through the C ABI.

The posterior factorises over independent spectrograms, so a batch must
give every job exactly the results it gets alone: the kernels treat frames
independently and chunk each job's chain from its own first frame, so the
comparison with a one-job context (same forward-backward chunk length) is
bit for bit.  Against the FP64 oracle the batch is held to the tolerances
of the single-job parity tests.
"""
import numpy as np
import pytest

from oracle import vi
from paper_1206_6468_gb300 import synth

pytestmark = pytest.mark.gpu

D_TOL = 1e-5
BOUND_RTOL = 1e-6


@pytest.fixture(scope="module")
def nf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def _jobs(lengths, seed=0, S=2, N=4, K=5, F=129, sigma=0.0):
    return synth.make_jobs(S, N, K, F, lengths, self_prob=0.9, energy_sigma=sigma, seed=seed)


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _alone(nf, jobs, j, chunk, precision="fp32", init_mode=0, V=None, fb_mode=0):
    """Job j in a context of its own, with the batch's forward-backward
    geometry (chunk, group): the same kernels' arithmetic for its frames."""
    V = _f32(jobs.V[j]) if V is None else V
    ctx = nf.VIContext(V, _f32(jobs.W), _f32(jobs.A), _f32(jobs.pi), jobs.S, jobs.N, jobs.K,
                       gamma=jobs.gamma, precision=precision, init_mode=init_mode)
    ctx.set_option("fb_chunk", chunk[0])
    ctx.set_option("fb_group", chunk[1])
    ctx.set_option("fb_mode", fb_mode)
    return ctx


def _geometry(ctx):
    return ctx.query("fb_chunk"), ctx.query("fb_group")


@pytest.mark.parametrize("precision", ["fp32", "bf16", "fp32_simt"])
@pytest.mark.parametrize("init_mode", [0, 1])
def test_batch_equals_each_job_alone(nf, precision, init_mode):
    lengths = [1, 5, 130, 777, 64, 300]
    jobs = _jobs(lengths, seed=11)
    with nf.VIContext(jobs.stacked_V(), _f32(jobs.W), _f32(jobs.A), _f32(jobs.pi), jobs.S,
                      jobs.N, jobs.K, precision=precision, init_mode=init_mode,
                      job_frames=lengths) as b:
        chunk = _geometry(b)
        total = b.sweep(4, bound=True)
        bounds = b.job_bounds()
        post = [b.job_posteriors(i) for i in b.job_ids]
        assert [j[2] for j in b.jobs()] == lengths
        assert all(j[3] == 4 for j in b.jobs())
    assert abs(total - bounds.sum()) <= 1e-12 * abs(total)
    for j in range(len(lengths)):
        with _alone(nf, jobs, j, chunk, precision, init_mode) as a:
            L = a.sweep(4, bound=True)
            d = a.posteriors()
        assert np.array_equal(post[j], d), f"job {j}"
        assert L == bounds[j], f"job {j}: {L} vs {bounds[j]}"


@pytest.mark.parametrize("fb_mode", [0, 4])
def test_batch_against_oracle(nf, fb_mode):
    """A three-job batch against the oracle run job by job (the scan, and the
    sequential forward-backward with four chains per block): the bound of
    every job after each of five sweeps (relative 1e-6), d-hat after the
    first sweep (1e-5, both sides starting from the same initial state) and
    after the fifth (1e-4: end to end, FP32 rounding at near-tie frames
    grows by a few times per sweep, as in the single-job trajectory tests),
    and the batch bound against the sum of the oracle's bounds."""
    lengths = [200, 37, 129]
    jobs = _jobs(lengths, seed=5)
    refs, first = [], []
    for j in range(len(lengths)):
        p = jobs.problem(j)
        V, W, A, pi = (x.astype(np.float32).astype(np.float64) for x in (p.V, p.W, p.A, p.pi))
        refs.append(vi.run(V, W, A, pi, p.S, p.N, p.K, p.gamma, 5))
        first.append(vi.run(V, W, A, pi, p.S, p.N, p.K, p.gamma, 1)["dhat"])
    with nf.VIContext(jobs.stacked_V(), _f32(jobs.W), _f32(jobs.A), _f32(jobs.pi), jobs.S,
                      jobs.N, jobs.K, job_frames=lengths) as b:
        b.set_option("fb_mode", fb_mode)
        assert b.query("fb_mode") == fb_mode
        Ls = []
        for i in range(5):
            b.sweep(1)
            Ls.append(b.job_bounds())
            if i == 0:
                post1 = [b.job_posteriors(k) for k in b.job_ids]
        post = [b.job_posteriors(k) for k in b.job_ids]
        L_total = b.bound()
    for j, ref in enumerate(refs):
        got = np.array([L[j] for L in Ls])
        assert np.all(np.abs(got - ref["bounds"]) <= BOUND_RTOL * np.abs(ref["bounds"])), j
        assert np.max(np.abs(post1[j] - first[j])) <= D_TOL, j
        assert np.max(np.abs(post[j] - ref["dhat"])) <= 10 * D_TOL, j
    want = sum(ref["bounds"][-1] for ref in refs)
    assert abs(L_total - want) <= BOUND_RTOL * abs(want)


@pytest.mark.parametrize("fb_mode", [0, 2])
def test_jobs_come_and_go(nf, fb_mode):
    """Add, sweep, remove from the middle, add again: every job's state is
    the one it has alone after the same number of sweeps (the scan, and the
    sequential forward-backward, whose blocks follow the job count)."""
    lengths = [90, 250, 33, 400]
    jobs = _jobs(lengths, seed=8, sigma=1.5)
    f = {k: _f32(getattr(jobs, k)) for k in ("W", "A", "pi")}
    with nf.Batch(f["W"], f["A"], f["pi"], jobs.S, jobs.N, jobs.K, capacity=500,
                  max_jobs=3) as b:
        chunk = _geometry(b)
        b.set_option("fb_mode", fb_mode)
        ids = [b.add(_f32(jobs.V[j])) for j in range(3)]
        b.sweep(3)
        b.remove(ids[1])                       # the frames of the third job move down
        with pytest.raises(nf.NfhmmError) as e:
            b.add(_f32(jobs.V[3]))             # 90 + 33 + 400 frames > 500
        assert e.value.code == nf.EFULL
        b.sweep(2)
        ids.append(b.add(np.ascontiguousarray(_f32(jobs.V[3])[:300])))   # 423 frames
        b.sweep(2)
        info = {j[0]: j for j in b.jobs()}
        assert [info[i][3] for i in (ids[0], ids[2], ids[3])] == [7, 7, 2]
        got = {i: b.job_posteriors(i) for i in (ids[0], ids[2], ids[3])}
        bounds = dict(zip([j[0] for j in b.jobs()], b.job_bounds()))
    for j, sweeps, idx in ((0, 7, 0), (2, 7, 2), (3, 2, 3)):
        V = np.ascontiguousarray(_f32(jobs.V[j])[:300]) if j == 3 else _f32(jobs.V[j])
        with _alone(nf, jobs, j, chunk, V=V, fb_mode=fb_mode) as a:
            L = a.sweep(sweeps, bound=True)
            d = a.posteriors()
        assert np.array_equal(got[ids[idx]], d), j
        # the batch's bound comes from a separate pass over alpha-hat after the
        # sweeps, the lone job's from sums formed during its last sweep: the
        # same quantity, rounded differently
        assert abs(bounds[ids[idx]] - L) <= 1e-8 * abs(L), j


def test_many_jobs_in_and_out_at_once(nf):
    """add_many, then remove_many of non-adjacent jobs (the survivors move
    down in one gather) and queued sweeps: each survivor and each newcomer
    equals its lone run bit for bit."""
    lengths = [40, 7, 130, 64, 1, 90, 55]
    jobs = _jobs(lengths, seed=13, sigma=1.0)
    f = {k: _f32(getattr(jobs, k)) for k in ("W", "A", "pi")}
    with nf.Batch(f["W"], f["A"], f["pi"], jobs.S, jobs.N, jobs.K, capacity=400,
                  max_jobs=6) as b:
        chunk = _geometry(b)
        assert b.query("frame_capacity") == 400 and b.query("max_jobs") == 6
        ids = b.add_many([_f32(jobs.V[j]) for j in range(5)])
        b.sweep_async(2)
        b.remove_many([ids[1], ids[3]])
        ids += b.add_many([_f32(jobs.V[5]), _f32(jobs.V[6])])
        b.sweep_async(3, prepare_bound=True)
        bounds = dict(zip([j[0] for j in b.jobs()], b.job_bounds()))
        got = {i: b.job_posteriors(i) for i in bounds}
        assert [j[2] for j in b.jobs()] == [40, 130, 1, 90, 55]
    for j, sweeps in ((0, 5), (2, 5), (4, 5), (5, 3), (6, 3)):
        with _alone(nf, jobs, j, chunk) as a:
            L = a.sweep(sweeps, bound=True)
            d = a.posteriors()
        assert np.array_equal(got[ids[j]], d), j
        assert bounds[ids[j]] == L, j


def test_batch_full_and_invalid_job_leave_batch_unchanged(nf):
    jobs = _jobs([100, 100], seed=2)
    f = {k: _f32(getattr(jobs, k)) for k in ("W", "A", "pi")}
    with nf.Batch(f["W"], f["A"], f["pi"], jobs.S, jobs.N, jobs.K, capacity=150,
                  max_jobs=4) as b:
        chunk = _geometry(b)
        i0 = b.add(_f32(jobs.V[0]))
        with pytest.raises(nf.NfhmmError) as e:
            b.add(_f32(jobs.V[1]))               # 200 frames > capacity 150
        assert e.value.code == nf.EFULL
        bad = np.ascontiguousarray(_f32(jobs.V[1])[:20])
        bad[3, 7] = -1.0
        with pytest.raises(nf.NfhmmError) as e:
            b.add(bad)
        assert e.value.code == nf.EINVAL
        assert [j[0] for j in b.jobs()] == [i0] and b.T == 100
        b.sweep(2)
        d = b.job_posteriors(i0)
    with _alone(nf, jobs, 0, chunk) as a:
        a.sweep(2)
        assert np.array_equal(a.posteriors(), d)


def test_empty_batch_sweeps_and_bound(nf):
    jobs = _jobs([10], seed=3)
    f = {k: _f32(getattr(jobs, k)) for k in ("W", "A", "pi")}
    with nf.Batch(f["W"], f["A"], f["pi"], jobs.S, jobs.N, jobs.K, capacity=64,
                  max_jobs=2) as b:
        assert b.sweep(2, bound=True) == 0.0
        i = b.add(_f32(jobs.V[0]))
        with pytest.raises(nf.NfhmmError) as e:
            b.bound()                             # no sweep since the job came
        assert e.value.code == nf.ESTATE
        b.sweep(1)
        b.remove(i)
        assert b.T == 0 and b.jobs() == []


def test_fb_options_change_only_rounding(nf):
    p = synth.make_problem(seed=4, **synth.SMALL)
    f = p.as_f32()
    out = []
    for L, prod in ((1, "simt"), (7, "tc"), (16, "simt"), (16, "tc"), (128, "simt")):
        with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
            ctx.set_option("fb_chunk", L)
            ctx.set_option("fb_products", prod)
            assert ctx.query("fb_chunk") == L
            out.append((ctx.sweep(3, bound=True), ctx.posteriors()))
    for L, d in out[1:]:
        assert abs(L - out[0][0]) <= 1e-7 * abs(out[0][0])
        assert np.max(np.abs(d - out[0][1])) <= 1e-5


def test_graph_replay_matches_direct_launches(nf):
    """Sweeps replayed from captured CUDA graphs equal sweeps launched one
    by one, also across job changes that invalidate the captured graph."""
    lengths = [120, 33, 260]
    jobs = _jobs(lengths, seed=17, sigma=1.0)
    f = {k: _f32(getattr(jobs, k)) for k in ("W", "A", "pi")}
    out = []
    for graphs in (1, 0):
        with nf.Batch(f["W"], f["A"], f["pi"], jobs.S, jobs.N, jobs.K, capacity=500,
                      max_jobs=3) as b:
            b.set_option("graphs", graphs)
            ids = b.add_many([_f32(v) for v in jobs.V[:2]])
            b.sweep(4)
            L1 = b.sweep(3, bound=True)
            b.remove(ids[0])
            ids.append(b.add(_f32(jobs.V[2])))
            b.sweep(4)
            L2 = b.sweep(2, bound=True)
            out.append((L1, L2, b.posteriors(), b.kernel_launches()))
    assert out[0][0] == out[1][0] and out[0][1] == out[1][1]
    assert np.array_equal(out[0][2], out[1][2])
    assert out[0][3] == out[1][3]


def test_profiling_through_graphs_counts_every_launch(nf):
    """With profiling on, sweeps replayed from a graph report the same stage
    invocations and launches as sweeps launched one by one."""
    p = synth.make_problem(seed=6, **synth.SMALL)
    f = p.as_f32()
    res = []
    for graphs in (1, 0):
        with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
            ctx.set_option("graphs", graphs)
            ctx.profile_enable(True)
            for _ in range(4):
                ctx.sweep(5, bound=True)
            prof = {st: ctx.profile_read(st) for st in ("weights", "gemm1", "gemm2", "fb",
                                                         "bound")}
            res.append((prof, ctx.posteriors()))
    for st in res[0][0]:
        ms_g, inv_g, l_g = res[0][0][st]
        ms_d, inv_d, l_d = res[1][0][st]
        assert inv_g == inv_d and l_g == l_d, st
        assert ms_g > 0 and ms_d > 0, st
    assert np.array_equal(res[0][1], res[1][1])


def test_multi_sweep_graphs_with_profiling_match_direct(nf):
    """Runs of plain sweeps replay from graphs of several sweeps, between the
    profiled sweeps (every 7th) and the run's last: the state, the bounds,
    the kernel launches and the stage invocations equal those of sweeps
    launched one by one."""
    lengths = [150, 77, 260]
    jobs = _jobs(lengths, seed=23, sigma=1.0)
    V, W, A, pi = (_f32(x) for x in (jobs.stacked_V(), jobs.W, jobs.A, jobs.pi))
    res = []
    for graphs in (1, 0):
        with nf.VIContext(V, W, A, pi, jobs.S, jobs.N, jobs.K, job_frames=lengths) as ctx:
            ctx.set_option("graphs", graphs)
            ctx.set_option("profile_stride", 7)
            ctx.profile_enable(True)
            Ls = [ctx.sweep(30, bound=True), ctx.sweep(11, bound=True)]
            ctx.profile_enable(False)
            Ls.append(ctx.sweep(19, bound=True))
            prof = {st: ctx.profile_read(st)[1:] for st in ("weights", "gemm1", "gemm2", "fb")}
            res.append((Ls, ctx.posteriors(), ctx.get_state()[0], ctx.kernel_launches(), prof))
    assert res[0][0] == res[1][0]
    assert np.array_equal(res[0][1], res[1][1]) and np.array_equal(res[0][2], res[1][2])
    assert res[0][3] == res[1][3]
    assert res[0][4] == res[1][4]


@pytest.mark.parametrize("where", ["pinned", "device"])
def test_inputs_read_in_place_equal_copied(nf, where):
    """Spectrograms in mapped pinned host memory or in device memory are read
    in place by the kernel that pads them into the frame store; pageable host
    memory is copied first: the same state either way, for a batch whose
    jobs lie back to back and for jobs added from buffers of their own."""
    import torch
    lengths = [300, 41, 777, 128]
    jobs = _jobs(lengths, seed=21, sigma=1.0)
    V, W, A, pi = (_f32(x) for x in (jobs.stacked_V(), jobs.W, jobs.A, jobs.pi))

    def place(x):
        t = torch.from_numpy(np.array(x, dtype=np.float32, copy=True))
        return t.pin_memory() if where == "pinned" else t.cuda()

    def run(Vx, Wx, Ax, pix):
        with nf.VIContext(Vx, Wx, Ax, pix, jobs.S, jobs.N, jobs.K, job_frames=lengths) as ctx:
            L = ctx.sweep(4, bound=True)
            return L, ctx.posteriors(), ctx.get_state()[0]

    ref = run(V, W, A, pi)
    got = run(*(place(x) for x in (V, W, A, pi)))
    assert got[0] == ref[0]
    assert np.array_equal(got[1], ref[1]) and np.array_equal(got[2], ref[2])
    out = []
    for per_job in ([_f32(v) for v in jobs.V], [place(v) for v in jobs.V]):
        with nf.Batch(W, A, pi, jobs.S, jobs.N, jobs.K, capacity=2000, max_jobs=8) as b:
            b.add_many(per_job)
            L = b.sweep(4, bound=True)
            out.append((L, b.posteriors()))
    assert out[0][0] == out[1][0] and np.array_equal(out[0][1], out[1][1])


def test_graphs_dropped_when_scratch_is_reallocated(nf):
    """A chunk length that needs more forward-backward scratch reallocates it;
    sweeps captured before then must not be replayed afterwards.  Going back
    to the first geometry (the same launch configuration as the first graphs)
    must give what launching one by one gives."""
    p = synth.make_problem(seed=9, **synth.SMALL)
    f = p.as_f32()
    out = []
    for graphs in (1, 0):
        with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
            ctx.set_option("graphs", graphs)
            L0 = ctx.query("fb_chunk")
            ctx.sweep(4)
            ctx.set_option("fb_chunk", 2)          # more chunks: new scratch
            ctx.sweep(3)
            ctx.set_option("fb_chunk", L0)
            out.append((ctx.sweep(4, bound=True), ctx.posteriors()))
    assert out[0][0] == out[1][0]
    assert np.array_equal(out[0][1], out[1][1])


@pytest.mark.parametrize("stride", [2, 3])
def test_profile_stride_times_every_kth_sweep(nf, stride):
    """With a profiling stride k, the stages of sweeps 0, k, 2k, ... of each
    run are timed, every launch is still counted, and results do not change."""
    p = synth.make_problem(seed=6, **synth.SMALL)
    f = p.as_f32()
    res = []
    for k in (1, stride):
        with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
            ctx.set_option("profile_stride", k)
            ctx.profile_enable(True)
            for _ in range(3):
                ctx.sweep(7, bound=True)
            prof = {st: ctx.profile_read(st) for st in ("weights", "fb")}
            res.append((prof, ctx.posteriors()))
    for st in ("weights", "fb"):
        assert res[0][0][st][1] == 3 * 7
        assert res[1][0][st][1] == 3 * len(range(0, 7, stride))
        assert res[0][0][st][2] == res[1][0][st][2]
    assert np.array_equal(res[0][1], res[1][1])


def test_autotune_picks_a_geometry_and_keeps_the_state(nf):
    """The autotuner times whole sweeps from a saved copy of the state: it
    needs a sweep, leaves posteriors and bound untouched, applies one of its
    candidates, and later sweeps equal those of a context set to that
    geometry and tile shape by hand at the same point (bit for bit: the same
    kernels run on the same state)."""
    p = synth.make_problem(seed=12, **synth.SMALL)
    f = p.as_f32()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
        with pytest.raises(nf.NfhmmError) as e:
            ctx.autotune()
        assert e.value.code == nf.ESTATE
        ctx.sweep(3)                       # no bound yet: the autotuner forms it first
        d0 = ctx.posteriors()
        r = ctx.autotune(reps=2)
        assert r["fb_chunk"] in (8, 12, 16, 20, 24, 32, 48, 64) and r["us"] > 0
        assert r["fb_mode"] in (0, 1, 2) and ctx.query("fb_mode") == r["fb_mode"]
        assert ctx.query("fb_chunk") == r["fb_chunk"]
        assert ctx.query("fb_group") == r["fb_group"]
        assert np.array_equal(ctx.posteriors(), d0)
        L0 = ctx.bound()
        L1, d1 = ctx.sweep(2, bound=True), ctx.posteriors()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ref:
        ref.sweep(3)
        L0r = ref.bound()
        ref.set_option("fb_chunk", r["fb_chunk"])
        ref.set_option("fb_group", r["fb_group"])
        ref.set_option("fb_mode", r["fb_mode"])
        t = r["tiles"]   # the tuner also chose the contractions' tile shapes
        ref.set_tiles(t["tile_gemm1"], t["tile_gemm2"], t["tile_stages1"], t["tile_stages2"],
                      t["tile_prefetch1"], t["tile_prefetch2"], t["tile_epi_stage1"],
                      t["tile_epi_stage2"])
        L1r, d1r = ref.sweep(2, bound=True), ref.posteriors()
    assert L0 == L0r
    assert L1 == L1r
    assert np.array_equal(d1, d1r)


@pytest.mark.parametrize("N, K", [(4, 5), (37, 3), (40, 2)])
def test_sequential_form_against_oracle(nf, N, K):
    """The sequential forward-backward against the oracle's forward-backward
    (Section 3.2) on the emissions of the first sweep: chains of 1 to 777
    frames (across the 32-frame emission blocks, ragged), one state per lane
    (N = 4) and two (N = 37, 40; 37 also takes the 4-byte copies of rows that
    are not 16-byte multiples).  After one sweep d-hat of every job is within
    1e-5 of the oracle's and the bound within 1e-6 relative; a batch with the
    scan form agrees to the same tolerances."""
    lengths = [1, 31, 32, 33, 64, 65, 130, 777]
    jobs = synth.make_jobs(2, N, K, 65, lengths, self_prob=0.9, energy_sigma=1.0, seed=21)
    refs = []
    for j in range(len(lengths)):
        p = jobs.problem(j)
        V, W, A, pi = (x.astype(np.float32).astype(np.float64) for x in (p.V, p.W, p.A, p.pi))
        refs.append(vi.run(V, W, A, pi, p.S, p.N, p.K, p.gamma, 1))
    out = {}
    for mode in (0, 8):
        with nf.VIContext(jobs.stacked_V(), _f32(jobs.W), _f32(jobs.A), _f32(jobs.pi), jobs.S,
                          jobs.N, jobs.K, job_frames=lengths) as b:
            b.set_option("fb_mode", mode)
            b.sweep(1)
            out[mode] = ([b.job_posteriors(k) for k in b.job_ids], b.job_bounds())
    for mode, (post, bounds) in out.items():
        for j, ref in enumerate(refs):
            assert np.max(np.abs(post[j] - ref["dhat"])) <= D_TOL, (mode, j)
            assert abs(bounds[j] - ref["bounds"][-1]) <= BOUND_RTOL * abs(ref["bounds"][-1]), (mode, j)
            assert np.allclose(post[j].sum(axis=-1), 1.0, atol=1e-5), (mode, j)


@pytest.mark.parametrize("precision", ["fp32", "bf16"])
def test_sequential_batch_equals_each_job_alone(nf, precision):
    """With the sequential form each chain's recursion, the d-hat pass and
    every contraction tile do the same arithmetic whatever else the batch
    holds or how many SMs the contractions keep: a batch and each job alone
    agree bit for bit."""
    lengths = [5, 130, 777, 64, 300]
    jobs = _jobs(lengths, seed=13)
    with nf.VIContext(jobs.stacked_V(), _f32(jobs.W), _f32(jobs.A), _f32(jobs.pi), jobs.S,
                      jobs.N, jobs.K, precision=precision, job_frames=lengths) as b:
        b.set_option("fb_mode", 2)
        b.sweep(3, bound=True)
        bounds = b.job_bounds()
        post = [b.job_posteriors(i) for i in b.job_ids]
    for j in range(len(lengths)):
        with _alone(nf, jobs, j, (16, 0), precision) as a:
            a.set_option("fb_mode", 2)
            L = a.sweep(3, bound=True)
            d = a.posteriors()
        assert np.array_equal(post[j], d), f"job {j}"
        assert L == bounds[j], f"job {j}: {L} vs {bounds[j]}"


def test_fb_mode_option_bounds(nf):
    p = synth.make_problem(seed=4, **synth.SMALL)
    f = p.as_f32()
    with nf.VIContext(f["V"], f["W"], f["A"], f["pi"], p.S, p.N, p.K) as ctx:
        assert ctx.query("fb_mode") == 0
        for bad in (-1, 65):
            with pytest.raises(nf.NfhmmError) as e:
                ctx.set_option("fb_mode", bad)
            assert e.value.code == nf.EINVAL
        ctx.set_option("fb_mode", 64)        # clamped to what a block holds
        assert 1 <= ctx.query("fb_mode") < 64
        L = ctx.sweep(2, bound=True)
        ctx.set_option("fb_mode", 0)
        assert ctx.query("fb_mode") == 0
    assert np.isfinite(L)


# ------------------------------------------- many tiles per persistent CTA

MANY_TILE_LENGTHS = [5000, 3001, 7000, 129, 4500, 900, 8000, 1, 2300]   # 30,831 frames


@pytest.fixture(scope="module")
def many_tile_case():
    """Nine jobs of uneven length on one S2 N40 K10 F513 model (the paper's
    sizes), and per job the oracle's state after one sweep (rounded to
    float32, as a context holds it) with the oracle's next sweep from it."""
    jobs = synth.make_jobs(2, 40, 10, 513, MANY_TILE_LENGTHS, self_prob=0.95, energy_sigma=1.5,
                           seed=21)
    jobs.W, jobs.A, jobs.pi = (x.astype(np.float32).astype(np.float64)
                               for x in (jobs.W, jobs.A, jobs.pi))
    B = vi.element_mask(jobs.S, jobs.N, jobs.K)
    states, refs = [], []
    for j in range(len(MANY_TILE_LENGTHS)):
        p = jobs.problem(j)
        V = p.V.astype(np.float32).astype(np.float64)
        c0, d0 = vi.init_state(V, p.W, p.S, p.N, p.K)
        st = vi.sweep(V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, c0, d0, B)
        c32, d32 = st["counts"].astype(np.float32), st["dhat"].astype(np.float32)
        ref = vi.sweep(V, p.W, p.A, p.pi, p.S, p.N, p.K, p.gamma, c32.astype(np.float64),
                       d32.astype(np.float64), B)
        ref["bound"] = vi.bound(V, p.W, ref["alpha"], ref["logZ"], p.gamma, p.S, p.K,
                                Vhat=ref["Vhat"])
        states.append((c32, d32))
        refs.append(ref)
    return jobs, states, refs


@pytest.mark.parametrize("fb_mode", [0, 4])
def test_many_tiles_per_cta_one_sweep_from_oracle_state(nf, many_tile_case, fb_mode):
    """A batch at the paper's sizes whose contractions walk several output
    tiles per persistent CTA: 30,831 frames give 241 row tiles, so 1,205
    reconstruction tiles (5 of 128 columns per row tile) and 1,446
    back-projection tiles (6 of 160) on at most 152 CTAs -- about 8-10 tiles
    each, through the TMEM hand-over between tiles and the stage ring that
    runs on across them; the sequential forward-backward (fb_mode 4) also
    takes SMs from their grid.  One sweep from the oracle's state after one
    sweep, every output of every job against the oracle's same sweep:
    alpha-hat, phi-hat (up to its per-frame constant) and counts element by
    element (2e-5 relative), d-hat (1e-5) and each job's bound (1e-6)."""
    from scipy.special import digamma as sp_digamma
    jobs, states, refs = many_tile_case
    counts = np.concatenate([c for c, _ in states], axis=0)
    dhat = np.concatenate([d for _, d in states], axis=1)
    with nf.VIContext(jobs.stacked_V(), _f32(jobs.W), _f32(jobs.A), _f32(jobs.pi), jobs.S,
                      jobs.N, jobs.K, job_frames=MANY_TILE_LENGTHS) as b:
        b.set_option("fb_mode", fb_mode)
        b.set_state(counts, dhat, 1)
        b.sweep(1)
        bounds = b.job_bounds()
        alpha = b.weights().astype(np.float64)
        phi = b.surrogate().astype(np.float64)
        counts_g, dhat_g, _ = b.get_state()
    t0 = 0
    for j, (T, ref) in enumerate(zip(MANY_TILE_LENGTHS, refs)):
        sl = slice(t0, t0 + T)
        t0 += T
        a = alpha[sl]
        assert np.max(np.abs(a - ref["alpha"]) / ref["alpha"]) <= 2e-5, j
        a0 = ref["alpha"].sum(axis=1)
        phi_ref = ref["phi"] + jobs.gamma * jobs.K * sp_digamma(a0)[None, :, None]
        assert np.max(np.abs(phi[:, sl] - phi_ref) / (1.0 + np.abs(phi_ref))) <= 2e-5, j
        c = counts_g[sl].astype(np.float64)
        big = ref["counts"] > 1e-2 * ref["counts"].max()
        assert np.max(np.abs(c[big] - ref["counts"][big]) / ref["counts"][big]) <= 2e-5, j
        assert np.max(np.abs(c - ref["counts"])) <= 2e-5 * ref["counts"].max(), j
        assert np.max(np.abs(dhat_g[:, sl] - ref["dhat"])) <= D_TOL, j
        assert abs(bounds[j] - ref["bound"]) <= BOUND_RTOL * abs(ref["bound"]), j
