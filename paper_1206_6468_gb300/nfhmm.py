"""ctypes binding of libnfhmm.so (the C ABI in include/nfhmm.h).

Argument marshalling only: every step of the sweep runs in the library's
CUDA kernels.  Host arrays are numpy float32 (C-contiguous); device arrays
are torch CUDA tensors (float32, contiguous), passed by data pointer, with
torch's current stream as the stream.  Importing this module loads the
library and raises ImportError if it has not been built.
"""
from __future__ import annotations

import ctypes
import os
import re
from typing import Optional

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "_lib", "libnfhmm.so")
HEADER_PATH = os.path.join(os.path.dirname(_HERE), "include", "nfhmm.h")

if not os.path.exists(LIB_PATH):
    raise ImportError(f"libnfhmm.so is not built ({LIB_PATH}); run __graft_entry__.build()")
_lib = ctypes.CDLL(LIB_PATH)

OK, EINVAL, ENOMEM, ECUDA, ETIMEOUT, ENUMERIC, ESTATE, EFULL = 0, -1, -2, -3, -4, -5, -6, -7
FP32, BF16, FP32_SIMT = 0, 1, 2
INIT_UNIFORM, INIT_PRIOR = 0, 1
SEP_MEAN, SEP_EXPECTATION = 0, 1
STAGES = {"weights": 0, "gemm1": 1, "gemm2": 2, "fb": 3, "bound": 4, "init": 5}
QUERIES = {"tensor_cores": 0, "fb_chunk": 1, "sweeps_done": 2, "device_bytes": 3,
           "frame_capacity": 4, "max_jobs": 5, "fb_group": 6, "fb_mode": 7, "tile_gemm1": 8,
           "tile_gemm2": 9, "tile_stages1": 10, "tile_stages2": 11, "tile_prefetch1": 12,
           "tile_prefetch2": 13, "tile_epi_stage1": 14, "tile_epi_stage2": 15}
OPTIONS = {"fb_chunk": 0, "fb_products": 1, "graphs": 2, "fb_group": 3, "profile_stride": 4,
           "fb_mode": 5, "test_wait_timeout": 6, "tile_gemm1": 7, "tile_gemm2": 8,
           "tile_stages1": 9, "tile_stages2": 10, "tile_prefetch1": 11, "tile_prefetch2": 12,
           "tile_epi_stage1": 13, "tile_epi_stage2": 14}
FB_PRODUCTS = {"simt": 0, "tc": 1}
PRECISIONS = {"fp32": FP32, "bf16": BF16, "fp32_simt": FP32_SIMT}


class Request(ctypes.Structure):
    _fields_ = [("model", ctypes.c_int), ("T", ctypes.c_int), ("V", ctypes.c_void_p),
                ("arrival_s", ctypes.c_double), ("dhat_out", ctypes.c_void_p)]


class ServeOpts(ctypes.Structure):
    _fields_ = [("rel_tol", ctypes.c_double), ("min_sweeps", ctypes.c_int),
                ("max_sweeps", ctypes.c_int), ("realtime", ctypes.c_int)]


class Result(ctypes.Structure):
    _fields_ = [("admit_s", ctypes.c_double), ("done_s", ctypes.c_double),
                ("sweeps", ctypes.c_int), ("bound", ctypes.c_double), ("status", ctypes.c_int)]


class Dims(ctypes.Structure):
    _fields_ = [("S", ctypes.c_int), ("N", ctypes.c_int), ("K", ctypes.c_int),
                ("F", ctypes.c_int), ("T", ctypes.c_int), ("gamma", ctypes.c_double),
                ("precision", ctypes.c_int), ("init_mode", ctypes.c_int)]


_vp = ctypes.c_void_p
_i = ctypes.c_int
_sigs = {
    "nfhmm_vi_init": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(Dims), _vp, _vp, _vp, _vp, _i, _vp]),
    "nfhmm_vi_reinit": (_i, [_vp, _vp, _vp, _vp, _vp, _i]),
    "nfhmm_vi_sweep": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double)]),
    "nfhmm_bound": (_i, [_vp, ctypes.POINTER(ctypes.c_double)]),
    "nfhmm_separate": (_i, [_vp, _vp, _i, _i, _i]),
    "nfhmm_get_posteriors": (_i, [_vp, _vp, _i]),
    "nfhmm_get_weights": (_i, [_vp, _vp, _i]),
    "nfhmm_get_surrogate": (_i, [_vp, _vp, _i]),
    "nfhmm_get_state": (_i, [_vp, _vp, _vp, ctypes.POINTER(_i), _i]),
    "nfhmm_set_state": (_i, [_vp, _vp, _vp, _i, _i]),
    "nfhmm_destroy": (None, [_vp]),
    "nfhmm_last_error": (ctypes.c_char_p, []),
    "nfhmm_forward_backward": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "nfhmm_forward_backward_noalloc": (_i, [_i, _i, _i, _vp, _vp, _vp, _vp, _vp, _i, _vp]),
    "nfhmm_digamma": (_i, [_vp, _vp, _vp, ctypes.c_size_t, _vp]),
    "nfhmm_mma_rate": (_i, [_i, ctypes.POINTER(ctypes.c_double), _vp]),
    "nfhmm_profile_enable": (_i, [_vp, _i]),
    "nfhmm_profile_read": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double),
                                ctypes.POINTER(ctypes.c_longlong),
                                ctypes.POINTER(ctypes.c_longlong), _i]),
    "nfhmm_query": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_longlong)]),
    "nfhmm_kernel_launches": (ctypes.c_longlong, [_vp]),
    "nfhmm_vi_init_batch": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(Dims), _i, _vp, _vp, _vp, _vp,
                                 _vp, _i, _vp, _vp]),
    "nfhmm_batch_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(Dims), _i, _vp, _vp, _vp, _i,
                                _vp]),
    "nfhmm_batch_add": (_i, [_vp, _i, _vp, _i, ctypes.POINTER(ctypes.c_longlong)]),
    "nfhmm_batch_remove": (_i, [_vp, ctypes.c_longlong]),
    "nfhmm_batch_add_many": (_i, [_vp, _i, _vp, _vp, _i, _vp]),
    "nfhmm_batch_remove_many": (_i, [_vp, _i, _vp]),
    "nfhmm_vi_sweep_async": (_i, [_vp, _i, _i]),
    "nfhmm_batch_info": (_i, [_vp, ctypes.POINTER(_i), ctypes.POINTER(_i), _vp, _vp, _vp, _vp]),
    "nfhmm_job_bounds": (_i, [_vp, _vp]),
    "nfhmm_job_posteriors": (_i, [_vp, ctypes.c_longlong, _vp, _i]),
    "nfhmm_set_option": (_i, [_vp, _i, ctypes.c_longlong]),
    "nfhmm_autotune": (_i, [_vp, _i, ctypes.POINTER(_i), ctypes.POINTER(_i),
                            ctypes.POINTER(ctypes.c_double)]),
    "nfhmm_serve": (_i, [ctypes.POINTER(_vp), _i, ctypes.POINTER(Request), _i,
                         ctypes.POINTER(ServeOpts), ctypes.POINTER(Result)]),
    "nfhmm_exact_create": (_i, [ctypes.POINTER(_vp), ctypes.POINTER(Dims), _vp, _vp, _vp, _vp, _i,
                                _vp]),
    "nfhmm_exact_iterate": (_i, [_vp, _i, ctypes.POINTER(ctypes.c_double)]),
    "nfhmm_exact_posteriors": (_i, [_vp, _vp, _i]),
    "nfhmm_exact_weights": (_i, [_vp, _vp, _i]),
    "nfhmm_exact_destroy": (None, [_vp]),
}
for _name, (_res, _args) in _sigs.items():
    _f = getattr(_lib, _name)
    _f.restype = _res
    _f.argtypes = _args


def declared_functions(header: str = HEADER_PATH):
    """Names of the functions include/nfhmm.h declares."""
    text = open(header).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(nfhmm_\w+)\s*\(", text)))


class NfhmmError(RuntimeError):
    def __init__(self, code: int, where: str):
        msg = _lib.nfhmm_last_error().decode()
        super().__init__(f"{where} failed with code {code}: {msg}")
        self.code = code


def _check(code: int, where: str):
    if code != OK:
        raise NfhmmError(code, where)


def _is_torch(x) -> bool:
    return type(x).__module__.startswith("torch")


def _ptr(x):
    """(pointer, on_device) of a numpy array or a torch tensor."""
    if _is_torch(x):
        import torch
        if x.dtype != torch.float32 and x.dtype != torch.float64:
            raise TypeError("tensors must be float32 (float64 for logZ)")
        if not x.is_contiguous():
            raise ValueError("tensors must be contiguous")
        return ctypes.c_void_p(x.data_ptr()), int(x.is_cuda)
    if not (isinstance(x, np.ndarray) and x.flags.c_contiguous):
        raise TypeError("host arrays must be C-contiguous numpy arrays")
    return ctypes.c_void_p(x.ctypes.data), 0


def _stream(stream=None):
    if stream is not None:
        return ctypes.c_void_p(int(stream))
    try:
        import torch
        if torch.cuda.is_available():
            return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    except Exception:  # pragma: no cover
        pass
    return ctypes.c_void_p(0)


def _f32(x):
    if _is_torch(x):
        return x
    return np.ascontiguousarray(x, dtype=np.float32)


def _model_ptrs(W, A, pi):
    ptrs = [_ptr(x) for x in (W, A, pi)]
    if len({d for _, d in ptrs}) != 1:
        raise ValueError("W, A, pi must all be on the host or all on the device")
    return [p for p, _ in ptrs], ptrs[0][1]


class VIContext:
    """Variational inference state on the GPU: one spectrogram, or a batch of
    jobs sharing one model (see Batch).

    V (T, F), W (M, F), A (S, N, N), pi (S, N): numpy arrays (host) or torch
    CUDA tensors (device), float32.  precision: "fp32" (split-TF32 tensor
    cores), "bf16" (BF16 tensor cores) or "fp32_simt" (FP32 CUDA cores)."""

    def __init__(self, V, W, A, pi, S: int, N: int, K: int, gamma: float = 1.0,
                 precision: str = "fp32", init_mode: int = INIT_UNIFORM, stream=None,
                 job_frames=None):
        V, W, A, pi = _f32(V), _f32(W), _f32(A), _f32(pi)
        T, F = V.shape
        self.S, self.N, self.K, self.F = S, N, K, F
        self.M = S * N * K
        self.gamma = gamma
        d = Dims(S, N, K, F, T, gamma, PRECISIONS[precision], init_mode)
        pv, dv = _ptr(V)
        (pw, pa, pp), dm = _model_ptrs(W, A, pi)
        if dv != dm:
            raise ValueError("V, W, A, pi must all be on the host or all on the device")
        h = ctypes.c_void_p()
        if job_frames is None:
            _check(_lib.nfhmm_vi_init(ctypes.byref(h), ctypes.byref(d), pv, pw, pa, pp, dv,
                                      _stream(stream)), "nfhmm_vi_init")
            self.job_ids = [0]
        else:
            fr = np.ascontiguousarray(job_frames, dtype=np.int32)
            ids = np.zeros(len(fr), dtype=np.int64)
            _check(_lib.nfhmm_vi_init_batch(ctypes.byref(h), ctypes.byref(d), len(fr),
                                            _vp(fr.ctypes.data), pv, pw, pa, pp, dv,
                                            _stream(stream), _vp(ids.ctypes.data)),
                   "nfhmm_vi_init_batch")
            self.job_ids = ids.tolist()
        self._h = h

    @property
    def T(self) -> int:
        """Frames held (all jobs)."""
        n, t = ctypes.c_int(), ctypes.c_int()
        _check(_lib.nfhmm_batch_info(self._h, ctypes.byref(n), ctypes.byref(t), None, None, None,
                                     None), "nfhmm_batch_info")
        return t.value

    def jobs(self):
        """List of (id, first frame, frames, sweeps) in frame order."""
        n, t = ctypes.c_int(), ctypes.c_int()
        _check(_lib.nfhmm_batch_info(self._h, ctypes.byref(n), ctypes.byref(t), None, None, None,
                                     None), "nfhmm_batch_info")
        ids = np.zeros(max(n.value, 1), dtype=np.int64)
        t0, T, sw = (np.zeros(max(n.value, 1), dtype=np.int32) for _ in range(3))
        _check(_lib.nfhmm_batch_info(self._h, ctypes.byref(n), ctypes.byref(t),
                                     _vp(ids.ctypes.data), _vp(t0.ctypes.data),
                                     _vp(T.ctypes.data), _vp(sw.ctypes.data)), "nfhmm_batch_info")
        return [(int(ids[j]), int(t0[j]), int(T[j]), int(sw[j])) for j in range(n.value)]

    def job_bounds(self) -> np.ndarray:
        n = len(self.jobs())
        out = np.zeros(max(n, 1), dtype=np.float64)
        _check(_lib.nfhmm_job_bounds(self._h, _vp(out.ctypes.data)), "nfhmm_job_bounds")
        return out[:n]

    def job_posteriors(self, job_id: int, out=None):
        T = {j[0]: j[2] for j in self.jobs()}[job_id]
        out = self._out((self.S, T, self.N), out)
        p, dev = _ptr(out)
        _check(_lib.nfhmm_job_posteriors(self._h, job_id, p, dev), "nfhmm_job_posteriors")
        return out

    def autotune(self, reps: int = 3) -> dict:
        """Time the forward-backward forms on the current jobs (after a sweep)
        and keep the fastest: {"fb_chunk", "fb_group", "fb_mode", "us"}
        (fb_mode 0: the scan over chunks; k >= 1: the sequential form, k
        chains per block)."""
        L, G, us = _i(), _i(), ctypes.c_double()
        _check(_lib.nfhmm_autotune(self._h, int(reps), ctypes.byref(L), ctypes.byref(G),
                                   ctypes.byref(us)), "nfhmm_autotune")
        out = {"fb_chunk": L.value, "fb_group": G.value, "fb_mode": self.query("fb_mode"),
               "us": us.value}
        if self.query("tensor_cores"):
            out["tiles"] = self.tiles()
        return out

    def tiles(self) -> dict:
        """The contractions' tile shapes: column tile and ring depth of each."""
        return {k: self.query(k) for k in ("tile_gemm1", "tile_gemm2", "tile_stages1",
                                           "tile_stages2", "tile_prefetch1", "tile_prefetch2",
                                           "tile_epi_stage1", "tile_epi_stage2")}

    def set_tiles(self, gemm1=None, gemm2=None, stages1=None, stages2=None, prefetch1=None,
                  prefetch2=None, epi_stage1=None, epi_stage2=None):
        # column tiles, then staging (it sets the deepest ring), then depths
        for k, v in (("tile_gemm1", gemm1), ("tile_gemm2", gemm2),
                     ("tile_epi_stage1", epi_stage1), ("tile_epi_stage2", epi_stage2),
                     ("tile_stages1", stages1), ("tile_stages2", stages2),
                     ("tile_prefetch1", prefetch1), ("tile_prefetch2", prefetch2)):
            if v is not None:
                self.set_option(k, v)

    def set_option(self, key: str, value):
        """fb_chunk: frames per chunk (1..128); fb_products: "simt" or "tc";
        fb_group: chunks per group (-1 automatic, 0 none); graphs: 0/1;
        profile_stride: time the stages of every k-th sweep of a run;
        fb_mode: 0 the scan over chunks, k >= 1 the sequential form with k
        chains per block; test_wait_timeout: ns, the failure-path test hook
        (NFHMM_OPT_TEST_WAIT_TIMEOUT); tile_gemm1, tile_gemm2: column tiles of
        the contractions; tile_stages1, tile_stages2: their ring depths."""
        if key == "fb_products":
            value = FB_PRODUCTS[value]
        _check(_lib.nfhmm_set_option(self._h, OPTIONS[key], int(value)), "nfhmm_set_option")

    def reinit(self, V, W, A, pi):
        """Load new inputs of the same sizes and reset to the initial state."""
        V, W, A, pi = _f32(V), _f32(W), _f32(A), _f32(pi)
        ptrs = [_ptr(x) for x in (V, W, A, pi)]
        if len({d for _, d in ptrs}) != 1:
            raise ValueError("V, W, A, pi must all be on the host or all on the device")
        _check(_lib.nfhmm_vi_reinit(self._h, *[p for p, _ in ptrs], ptrs[0][1]),
               "nfhmm_vi_reinit")

    # -- sweeps and bound
    def sweep(self, n: int = 1, bound: bool = False) -> Optional[float]:
        if bound:
            out = ctypes.c_double()
            _check(_lib.nfhmm_vi_sweep(self._h, n, ctypes.byref(out)), "nfhmm_vi_sweep")
            return out.value
        _check(_lib.nfhmm_vi_sweep(self._h, n, None), "nfhmm_vi_sweep")
        return None

    def sweep_async(self, n: int = 1, prepare_bound: bool = False):
        """Queue n sweeps without waiting (see nfhmm_vi_sweep_async)."""
        _check(_lib.nfhmm_vi_sweep_async(self._h, n, int(prepare_bound)), "nfhmm_vi_sweep_async")

    def bound(self) -> float:
        out = ctypes.c_double()
        _check(_lib.nfhmm_bound(self._h, ctypes.byref(out)), "nfhmm_bound")
        return out.value

    # -- outputs
    def _out(self, shape, out):
        if out is None:
            out = np.empty(shape, dtype=np.float32)
        if tuple(out.shape) != tuple(shape):
            raise ValueError(f"output must have shape {shape}")
        return out

    def separate(self, masked: bool = True, weights: str = "mean", out=None):
        out = self._out((self.S, self.T, self.F), out)
        p, dev = _ptr(out)
        _check(_lib.nfhmm_separate(self._h, p, int(masked),
                                   {"mean": SEP_MEAN, "expectation": SEP_EXPECTATION}[weights],
                                   dev), "nfhmm_separate")
        return out

    def posteriors(self, out=None):
        out = self._out((self.S, self.T, self.N), out)
        p, dev = _ptr(out)
        _check(_lib.nfhmm_get_posteriors(self._h, p, dev), "nfhmm_get_posteriors")
        return out

    def weights(self, out=None):
        out = self._out((self.T, self.M), out)
        p, dev = _ptr(out)
        _check(_lib.nfhmm_get_weights(self._h, p, dev), "nfhmm_get_weights")
        return out

    def surrogate(self, out=None):
        out = self._out((self.S, self.T, self.N), out)
        p, dev = _ptr(out)
        _check(_lib.nfhmm_get_surrogate(self._h, p, dev), "nfhmm_get_surrogate")
        return out

    def get_state(self):
        counts = np.empty((self.T, self.M), dtype=np.float32)
        dhat = np.empty((self.S, self.T, self.N), dtype=np.float32)
        n = ctypes.c_int()
        _check(_lib.nfhmm_get_state(self._h, _ptr(counts)[0], _ptr(dhat)[0], ctypes.byref(n), 0),
               "nfhmm_get_state")
        return counts, dhat, n.value

    def set_state(self, counts, dhat, sweeps_done: int = 0):
        counts, dhat = _f32(counts), _f32(dhat)
        pc, dc = _ptr(counts)
        pd, dd = _ptr(dhat)
        if dc != dd:
            raise ValueError("counts and dhat must be on the same side")
        _check(_lib.nfhmm_set_state(self._h, pc, pd, sweeps_done, dc), "nfhmm_set_state")

    # -- profiling
    def profile_enable(self, on: bool = True):
        _check(_lib.nfhmm_profile_enable(self._h, int(on)), "nfhmm_profile_enable")

    def profile_read(self, stage: str, reset: bool = False):
        """(summed event ms, stage invocations, kernel launches) of one stage."""
        ms = ctypes.c_double()
        inv = ctypes.c_longlong()
        n = ctypes.c_longlong()
        _check(_lib.nfhmm_profile_read(self._h, STAGES[stage], ctypes.byref(ms), ctypes.byref(inv),
                                       ctypes.byref(n), int(reset)), "nfhmm_profile_read")
        return ms.value, inv.value, n.value

    def query(self, key: str) -> int:
        v = ctypes.c_longlong()
        _check(_lib.nfhmm_query(self._h, QUERIES[key], ctypes.byref(v)), "nfhmm_query")
        return v.value

    def kernel_launches(self) -> int:
        return int(_lib.nfhmm_kernel_launches(self._h))

    def close(self):
        if getattr(self, "_h", None):
            _lib.nfhmm_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


class Batch(VIContext):
    """An empty batch with room for `capacity` frames and `max_jobs` jobs that
    share one model; jobs are added and removed between sweeps."""

    def __init__(self, W, A, pi, S: int, N: int, K: int, capacity: int, max_jobs: int,
                 gamma: float = 1.0, precision: str = "fp32", init_mode: int = INIT_UNIFORM,
                 stream=None):
        W, A, pi = _f32(W), _f32(A), _f32(pi)
        F = W.shape[1]
        self.S, self.N, self.K, self.F = S, N, K, F
        self.M = S * N * K
        self.gamma = gamma
        self.capacity, self.max_jobs = capacity, max_jobs
        d = Dims(S, N, K, F, capacity, gamma, PRECISIONS[precision], init_mode)
        (pw, pa, pp), dm = _model_ptrs(W, A, pi)
        h = ctypes.c_void_p()
        _check(_lib.nfhmm_batch_create(ctypes.byref(h), ctypes.byref(d), max_jobs, pw, pa, pp, dm,
                                       _stream(stream)), "nfhmm_batch_create")
        self._h = h
        self.job_ids = []

    def add(self, V) -> int:
        """Append a job (V: (T, F)); returns its id.  Raises NfhmmError with
        code EFULL when the batch has no room."""
        V = _f32(V)
        p, dev = _ptr(V)
        jid = ctypes.c_longlong()
        _check(_lib.nfhmm_batch_add(self._h, V.shape[0], p, dev, ctypes.byref(jid)),
               "nfhmm_batch_add")
        return jid.value

    def remove(self, job_id: int):
        _check(_lib.nfhmm_batch_remove(self._h, job_id), "nfhmm_batch_remove")

    def add_many(self, Vs) -> list:
        """Append several jobs at once (validated together); returns their ids."""
        Vs = [_f32(V) for V in Vs]
        ptrs = [_ptr(V) for V in Vs]
        if len({d for _, d in ptrs}) > 1:
            raise ValueError("all spectrograms on the host or all on the device")
        n = len(Vs)
        T = np.array([V.shape[0] for V in Vs], dtype=np.int32)
        arr = (_vp * max(n, 1))(*[p.value for p, _ in ptrs])
        ids = np.zeros(max(n, 1), dtype=np.int64)
        _check(_lib.nfhmm_batch_add_many(self._h, n, _vp(T.ctypes.data), arr,
                                         ptrs[0][1] if n else 0, _vp(ids.ctypes.data)),
               "nfhmm_batch_add_many")
        return ids[:n].tolist()

    def remove_many(self, job_ids):
        ids = np.ascontiguousarray(job_ids, dtype=np.int64)
        _check(_lib.nfhmm_batch_remove_many(self._h, len(ids), _vp(ids.ctypes.data)),
               "nfhmm_batch_remove_many")


class ExactNFHMM:
    """Exact inference in the original N-FHMM (the comparison system):
    per-(frame, joint state) weights, EM with forward-backward over the N^S
    joint states.  Same input conventions as VIContext."""

    def __init__(self, V, W, A, pi, S: int, N: int, K: int, precision: str = "fp32",
                 stream=None):
        V, W, A, pi = _f32(V), _f32(W), _f32(A), _f32(pi)
        T, F = V.shape
        self.S, self.N, self.K, self.F, self.T = S, N, K, F, T
        self.NC = N ** S
        d = Dims(S, N, K, F, T, 1.0, PRECISIONS[precision], 0)
        ptrs = [_ptr(x) for x in (V, W, A, pi)]
        if len({dv for _, dv in ptrs}) != 1:
            raise ValueError("V, W, A, pi must all be on the host or all on the device")
        h = ctypes.c_void_p()
        _check(_lib.nfhmm_exact_create(ctypes.byref(h), ctypes.byref(d), *[p for p, _ in ptrs],
                                       ptrs[0][1], _stream(stream)), "nfhmm_exact_create")
        self._h = h

    def iterate(self, n: int = 1, loglik: bool = True) -> Optional[float]:
        if loglik:
            out = ctypes.c_double()
            _check(_lib.nfhmm_exact_iterate(self._h, n, ctypes.byref(out)), "nfhmm_exact_iterate")
            return out.value
        _check(_lib.nfhmm_exact_iterate(self._h, n, None), "nfhmm_exact_iterate")
        return None

    def posteriors(self, out=None):
        out = np.empty((self.T, self.NC), dtype=np.float32) if out is None else out
        p, dev = _ptr(out)
        _check(_lib.nfhmm_exact_posteriors(self._h, p, dev), "nfhmm_exact_posteriors")
        return out

    def weights(self, out=None):
        out = np.empty((self.T, self.NC, self.S * self.K), dtype=np.float32) if out is None else out
        p, dev = _ptr(out)
        _check(_lib.nfhmm_exact_weights(self._h, p, dev), "nfhmm_exact_weights")
        return out

    def close(self):
        if getattr(self, "_h", None):
            _lib.nfhmm_exact_destroy(self._h)
            self._h = None

    def __del__(self):
        self.close()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()


def serve(batches, requests, rel_tol: float = 1e-5, min_sweeps: int = 2,
          max_sweeps: int = 100, realtime: bool = True, want_posteriors: bool = True):
    """Run nfhmm_serve.  batches: empty Batch objects (one per model);
    requests: list of (model index, V (T, F) numpy float32, arrival seconds).
    Returns (results as a list of dicts, posteriors per request or None)."""
    n = len(requests)
    reqs = (Request * max(n, 1))()
    keep, outs = [], []
    for r, (m, V, t) in enumerate(requests):
        V = np.ascontiguousarray(V, dtype=np.float32)
        b = batches[m]
        out = np.empty((b.S, V.shape[0], b.N), dtype=np.float32) if want_posteriors else None
        keep.append(V)
        outs.append(out)
        reqs[r] = Request(m, V.shape[0], V.ctypes.data, float(t),
                          out.ctypes.data if out is not None else None)
    handles = (_vp * len(batches))(*[b._h.value for b in batches])
    opts = ServeOpts(rel_tol, min_sweeps, max_sweeps, int(realtime))
    res = (Result * max(n, 1))()
    _check(_lib.nfhmm_serve(handles, len(batches), reqs, n, ctypes.byref(opts), res),
           "nfhmm_serve")
    results = [dict(admit_s=res[r].admit_s, done_s=res[r].done_s, sweeps=res[r].sweeps,
                    bound=res[r].bound, status=res[r].status) for r in range(n)]
    return results, outs


def forward_backward(phi, A, pi, chunk_len: int = 0, stream=None):
    """d-hat and log Z of S independent chains (torch CUDA tensors in/out)."""
    import torch
    S, T, N = phi.shape
    dhat = torch.empty_like(phi)
    logZ = torch.empty(S, dtype=torch.float64, device=phi.device)
    _check(_lib.nfhmm_forward_backward(S, N, T, _ptr(phi)[0], _ptr(A)[0], _ptr(pi)[0],
                                       _ptr(dhat)[0], _ptr(logZ)[0], chunk_len, _stream(stream)),
           "nfhmm_forward_backward")
    return dhat, logZ


def digamma(x, stream=None):
    """(psi(x), exp(psi(x))) from the library's device digamma (torch CUDA tensors)."""
    import torch
    psi = torch.empty_like(x)
    w = torch.empty_like(x)
    _check(_lib.nfhmm_digamma(_ptr(x)[0], _ptr(psi)[0], _ptr(w)[0], x.numel(), _stream(stream)),
           "nfhmm_digamma")
    return psi, w


def mma_rate(precision: str = "fp32", stream=None) -> float:
    """Measured dense tensor-core rate in TFLOP/s for the operand kind of a
    precision (fp32: one tf32 pass; bf16) -- see nfhmm_mma_rate."""
    out = ctypes.c_double()
    _check(_lib.nfhmm_mma_rate(PRECISIONS[precision], ctypes.byref(out), _stream(stream)),
           "nfhmm_mma_rate")
    return out.value


def call_raw(name: str):
    """The raw ctypes function (for tests of the ABI's error handling)."""
    return getattr(_lib, name)
