"""Continuous batching (nfhmm_serve) through the C ABI.

A request's result must be the same served alone and served in a mix of
requests of two models that come and go: the posterior factorises over
requests, the kernels treat frames independently and each request's chain
is chunked from its own first frame, so the comparison is bit for bit
(same batch geometry, hence the same forward-backward chunk length).
"""
import numpy as np
import pytest

from oracle import vi
from paper_1206_6468_gb300 import synth

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def nf():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def _f32(x):
    return np.ascontiguousarray(x, dtype=np.float32)


def _models():
    a = synth.make_jobs(2, 4, 5, 129, [60, 300, 17, 200, 90], self_prob=0.9, energy_sigma=1.0,
                        seed=21)
    b = synth.make_jobs(3, 3, 4, 129, [150, 33, 240], self_prob=0.9, energy_sigma=1.0, seed=22)
    return [a, b]


def _batches(nf, models, capacity=400, max_jobs=3):
    return [nf.Batch(_f32(m.W), _f32(m.A), _f32(m.pi), m.S, m.N, m.K, capacity=capacity,
                     max_jobs=max_jobs) for m in models]


def _requests(models):
    reqs = []
    for mi, m in enumerate(models):
        for j, V in enumerate(m.V):
            reqs.append((mi, _f32(V), 0.001 * (len(reqs))))
    return reqs


def test_serve_same_alone_and_in_mix(nf):
    models = _models()
    reqs = _requests(models)
    bs = _batches(nf, models)
    try:
        res, post = nf.serve(bs, reqs, rel_tol=1e-5, max_sweeps=40, realtime=False)
    finally:
        for b in bs:
            b.close()
    assert all(r["status"] == nf.OK for r in res)
    assert all(2 <= r["sweeps"] <= 40 for r in res)
    # the mix had to queue: capacity 400 frames, 3 slots per model
    assert max(r["admit_s"] for r in res) > min(r["done_s"] for r in res)
    for i, (mi, V, _) in enumerate(reqs):
        bs = _batches(nf, models)
        try:
            r1, p1 = nf.serve(bs, [(mi, V, 0.0)], rel_tol=1e-5, max_sweeps=40, realtime=False)
        finally:
            for b in bs:
                b.close()
        assert r1[0]["sweeps"] == res[i]["sweeps"], i
        assert r1[0]["bound"] == res[i]["bound"], i
        assert np.array_equal(p1[0], post[i]), i


def test_served_request_matches_oracle(nf):
    """Six sweeps of two served requests against the oracle's six sweeps:
    the bound to 1e-6 relative; d-hat to 1e-4, the end-to-end allowance
    (FP32 rounding at near-tie frames grows by a few times per sweep; the
    strict 1e-5 check of a single sweep from the oracle's state is in the
    single-job parity tests)."""
    models = _models()
    reqs = _requests(models)
    bs = _batches(nf, models)
    try:
        res, post = nf.serve(bs, reqs, rel_tol=1e-5, max_sweeps=6, min_sweeps=6,
                             realtime=False)
    finally:
        for b in bs:
            b.close()
    for i in (0, 6):
        mi, V, _ = reqs[i]
        m = models[mi]
        W, A, pi = (x.astype(np.float32).astype(np.float64) for x in (m.W, m.A, m.pi))
        ref = vi.run(V.astype(np.float64), W, A, pi, m.S, m.N, m.K, m.gamma, 6)
        assert res[i]["sweeps"] == 6
        assert abs(res[i]["bound"] - ref["bounds"][-1]) <= 1e-6 * abs(ref["bounds"][-1])
        assert np.max(np.abs(post[i] - ref["dhat"])) <= 1e-4


def test_serve_realtime_and_oversized_request(nf):
    models = _models()
    reqs = [(0, _f32(models[0].V[0]), 0.0), (1, _f32(models[1].V[1]), 0.05),
            (0, _f32(np.concatenate(models[0].V[:3])), 0.02),      # 377 frames: fits
            (1, _f32(np.concatenate(models[1].V)), 0.03)]          # 423 > 400 frames: never fits
    bs = _batches(nf, models)
    try:
        res, post = nf.serve(bs, reqs, rel_tol=1e-4, max_sweeps=20, realtime=True)
    finally:
        for b in bs:
            b.close()
    assert res[3]["status"] == nf.EFULL
    for r, (_, _, t) in zip(res[:3], reqs[:3]):
        assert r["status"] == nf.OK
        assert r["admit_s"] >= t and r["done_s"] > r["admit_s"]
    for p in post[:3]:
        assert np.allclose(p.sum(axis=2), 1.0, atol=1e-5)
