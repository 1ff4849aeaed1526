"""The allocation-free forward-backward entry point.

Callers that must not allocate device memory when they call in (a runtime
that owns a fixed HBM budget, a latency-critical thread that cannot risk a
blocking cudaMalloc) use nfhmm_forward_backward_noalloc, whose scratch lives
in a fixed device array inside the library.  Called through the C ABI, its
results must equal those of nfhmm_forward_backward (which allocates its
scratch on the stream) within the forward-backward tolerance of the parity
tests, on two calls in a row (the array keeps the previous call's contents).
This file is collected last on purpose; it also passes alone in a fresh
process.
"""
import ctypes

import numpy as np
import pytest

pytestmark = pytest.mark.gpu

D_TOL = 1e-5


@pytest.fixture(scope="module")
def lib():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def _inputs(seed, S, N, T, scale):
    import torch
    from paper_1206_6468_gb300 import synth
    rng = np.random.default_rng(seed)
    A = np.stack([0.5 * rng.dirichlet(np.ones(N), size=N) + 0.5 * synth.transition_matrix(N, 0.9)
                  for _ in range(S)]).astype(np.float32)
    pi = rng.dirichlet(np.ones(N), size=S).astype(np.float32)
    phi = (scale * rng.standard_normal((S, T, N))).astype(np.float32)
    return [torch.from_numpy(x).cuda() for x in (phi, A, pi)]


def _call(lib, name, phi, A, pi, chunk_len, stream):
    import torch
    S, T, N = phi.shape
    dhat = torch.full_like(phi, -1.0)
    logZ = torch.full((S,), -1.0, dtype=torch.float64, device=phi.device)
    fn = lib.call_raw(name)
    rc = fn(S, N, T, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(A.data_ptr()),
            ctypes.c_void_p(pi.data_ptr()), ctypes.c_void_p(dhat.data_ptr()),
            ctypes.c_void_p(logZ.data_ptr()), chunk_len, ctypes.c_void_p(stream))
    assert rc == lib.OK, lib._lib.nfhmm_last_error().decode()
    return dhat, logZ


@pytest.mark.parametrize("S,N,T,L,scale", [(2, 40, 3000, 0, 20.0), (3, 7, 130, 16, 10.0)])
def test_noalloc_matches_allocating_entry_point(lib, S, N, T, L, scale):
    import torch
    stream = torch.cuda.current_stream().cuda_stream
    for call in range(2):
        phi, A, pi = _inputs(100 * call + S + N + T, S, N, T, scale)
        d_ref, z_ref = _call(lib, "nfhmm_forward_backward", phi, A, pi, L, stream)
        d_na, z_na = _call(lib, "nfhmm_forward_backward_noalloc", phi, A, pi, L, stream)
        torch.cuda.synchronize()
        d_ref, z_ref = d_ref.cpu().numpy(), z_ref.cpu().numpy()
        d_na, z_na = d_na.cpu().numpy(), z_na.cpu().numpy()
        assert np.max(np.abs(d_na - d_ref)) <= D_TOL
        assert np.all(np.abs(z_na - z_ref) <= 1e-6 * np.maximum(1.0, np.abs(z_ref)))
        assert np.allclose(d_na.sum(axis=2), 1.0, atol=1e-5)


def test_noalloc_rejects_oversized_problem(lib):
    import torch
    S, N, T = 4, 64, 60000          # chunk matrices alone exceed the fixed array
    phi = torch.zeros((S, T, N), dtype=torch.float32, device="cuda")
    A = torch.full((S, N, N), 1.0 / N, dtype=torch.float32, device="cuda")
    pi = torch.full((S, N), 1.0 / N, dtype=torch.float32, device="cuda")
    out = torch.empty_like(phi)
    logZ = torch.empty(S, dtype=torch.float64, device="cuda")
    fn = lib.call_raw("nfhmm_forward_backward_noalloc")
    rc = fn(S, N, T, ctypes.c_void_p(phi.data_ptr()), ctypes.c_void_p(A.data_ptr()),
            ctypes.c_void_p(pi.data_ptr()), ctypes.c_void_p(out.data_ptr()),
            ctypes.c_void_p(logZ.data_ptr()), 0, ctypes.c_void_p(0))
    assert rc == lib.EINVAL
    assert "bytes of scratch" in lib._lib.nfhmm_last_error().decode()


def test_noalloc_reports_zero_probability_then_recovers(lib):
    """A device-side failure (here data of probability zero under one chain:
    an emission excludes the only state its transitions allow) turns every
    log normaliser into NaN; the array keeps that call's error word, and the
    next call clears it and gives the allocating entry point's results."""
    import torch
    from test_gpu_failure import zero_probability_inputs
    stream = torch.cuda.current_stream().cuda_stream
    phi, A, pi = zero_probability_inputs()
    _, z_bad = _call(lib, "nfhmm_forward_backward_noalloc", phi, A, pi, 0, stream)
    torch.cuda.synchronize()
    assert torch.isnan(z_bad).all()
    phi, A, pi = (x[:1].contiguous() for x in (phi, A, pi))
    d_ref, z_ref = _call(lib, "nfhmm_forward_backward", phi, A, pi, 0, stream)
    d_na, z_na = _call(lib, "nfhmm_forward_backward_noalloc", phi, A, pi, 0, stream)
    torch.cuda.synchronize()
    assert torch.isfinite(z_na).all()
    assert float((d_na - d_ref).abs().max()) <= D_TOL
    assert float((z_na - z_ref).abs().max()) <= 1e-6 * max(1.0, float(z_ref.abs().max()))
