"""The C-ABI library builds (nvcc cross-compiles sm_103a), loads without a
GPU, exports every function include/nfhmm.h declares, and rejects bad
arguments on the host before touching the device."""
import ctypes

import pytest


@pytest.fixture(scope="module")
def lib():
    from paper_1206_6468_gb300 import build
    build.build()
    from paper_1206_6468_gb300 import nfhmm
    return nfhmm


def test_exports_every_declared_function(lib):
    names = lib.declared_functions()
    assert len(names) >= 16
    missing = [n for n in names if not hasattr(lib._lib, n)]
    assert not missing, missing


def test_null_arguments_rejected(lib):
    init = lib.call_raw("nfhmm_vi_init")
    h = ctypes.c_void_p()
    d = lib.Dims(2, 4, 5, 129, 200, 1.0, 0, 0)
    assert init(ctypes.byref(h), ctypes.byref(d), None, None, None, None, 0, None) == lib.EINVAL
    assert h.value is None
    assert "NULL" in lib._lib.nfhmm_last_error().decode()
    assert lib.call_raw("nfhmm_vi_sweep")(None, 1, None) == lib.EINVAL
    out = ctypes.c_double()
    assert lib.call_raw("nfhmm_bound")(None, ctypes.byref(out)) == lib.EINVAL
    assert lib.call_raw("nfhmm_separate")(None, None, 1, 0, 0) == lib.EINVAL
    assert lib.call_raw("nfhmm_get_posteriors")(None, None, 0) == lib.EINVAL
    assert lib.call_raw("nfhmm_forward_backward")(1, 2, 3, None, None, None, None, None, 0,
                                                  None) == lib.EINVAL
    assert lib.call_raw("nfhmm_kernel_launches")(None) == 0
    lib.call_raw("nfhmm_destroy")(None)


@pytest.mark.parametrize("dims,msg", [
    ((0, 4, 5, 129, 200, 1.0, 0, 0), ">= 1"),
    ((2, 4, 5, 129, 0, 1.0, 0, 0), ">= 1"),
    ((2, 65, 5, 129, 200, 1.0, 0, 0), "N must be"),
    ((2, 4, 5, 129, 200, -1.0, 0, 0), "gamma"),
    ((2, 4, 5, 129, 200, 1.0, 7, 0), "precision"),
    ((2, 4, 5, 129, 200, 1.0, 0, 9), "init_mode"),
])
def test_bad_dims_rejected(lib, dims, msg):
    import numpy as np
    buf = np.zeros(16, dtype=np.float32)
    p = ctypes.c_void_p(buf.ctypes.data)
    h = ctypes.c_void_p()
    d = lib.Dims(*dims)
    rc = lib.call_raw("nfhmm_vi_init")(ctypes.byref(h), ctypes.byref(d), p, p, p, p, 0, None)
    assert rc == lib.EINVAL
    assert msg in lib._lib.nfhmm_last_error().decode()


def _header_defines(prefix):
    import re
    from paper_1206_6468_gb300 import nfhmm
    text = open(nfhmm.HEADER_PATH).read()
    return {m.group(1): int(m.group(2))
            for m in re.finditer(r"#define\s+(" + prefix + r"\w+)\s+(-?\d+)", text)}


def test_binding_option_and_query_codes_match_the_header(lib):
    """The ctypes binding's names for nfhmm_set_option / nfhmm_query keys are
    the header's values (a key added on one side only would silently set or
    read the wrong property)."""
    opts = _header_defines("NFHMM_OPT_")
    qs = _header_defines("NFHMM_Q_")
    assert {k.lower().replace("nfhmm_opt_", ""): v for k, v in opts.items()} == lib.OPTIONS
    assert {k.lower().replace("nfhmm_q_", ""): v for k, v in qs.items()} == lib.QUERIES


def test_bench_forward_backward_critical_path_model():
    """Serial frame steps on the forward-backward's critical path, as the
    bench reports them: the longest chain for the sequential form; a chunk
    twice plus the scan across chunks (or groups) for the scan."""
    import importlib.util, os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.fb_serial_steps(7993, 2, 64, 0) == (7993, "sequential")
    assert bench.fb_serial_steps(3000, 0, 12, 12) == (2 * 12 + 12 + 21, "scan")   # 250 chunks
    assert bench.fb_serial_steps(3000, 0, 32, 0) == (2 * 32 + 94, "scan")          # 94 chunks


def test_bench_tensor_peaks_and_split_tf32_ceiling():
    """The contractions' roofline denominators: the tf32 rate measured in the
    run when there is one (else bf16 sustained x the nominal tf32/bf16
    ratio), bf16 from the measured peaks; the split-TF32 form issues three
    tf32 MMAs per product, so its ceiling is a third of the tf32 peak."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod2", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    peaks = bench.load_peaks({"tf32": 1300.0, "bf16": 2500.0})
    pk, note = bench.tensor_peak("fp32", peaks)
    assert pk == 1300.0 and "measured in this run" in note
    assert bench.tensor_peak("bf16", peaks)[0] == peaks["bf16_tflops_sustained"]
    no_probe = bench.load_peaks(None)
    assert bench.tensor_peak("fp32", no_probe)[0] == no_probe["bf16_tflops_sustained"] * 1.1 / 2.25
    # one launch of 0.1 ms per stage; 2 T F M flops per contraction launch
    prof = {"weights": (1.0, 10, 10), "gemm1": (1.0, 10, 10), "gemm2": (1.0, 10, 10),
            "fb": (1.0, 10, 50)}
    r = bench.stage_rooflines(prof, 3000, 2, 40, 10, 513, "fp32", True, peaks, (57, "scan"))
    achieved = 2.0 * 3000 * 513 * 800 / 1e-4 / 1e12
    assert abs(r["gemm1"]["achieved"] - round(achieved, 2)) < 1e-9
    assert r["gemm1"]["split_tf32_ceiling"] == round(1300.0 / 3, 1)
    assert abs(r["gemm1"]["frac_of_split_ceiling"] - round(3 * achieved / 1300.0, 4)) < 1e-9
    assert r["fb"]["critical_path"]["ns_per_step"] == round(1e5 / 57, 1)
    dom = bench.roofline_of(prof, 3000, 2, 40, 10, 513, "fp32", True, peaks, 10,
                            fb_path=(57, "scan"))
    assert dom["kernel"] in prof and dom["peak"] > 0


def test_bench_traffic_summary_is_keyed_to_the_sources(monkeypatch):
    """The committed DRAM-traffic summary carries every stage and the hash of
    the library sources it was captured from; the bench reports its figures
    only while the sources still hash to that value."""
    import importlib.util
    import os
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    spec = importlib.util.spec_from_file_location("bench_mod3", os.path.join(root, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    text = open(os.path.join(root, "profiles", "traffic_paper_size_fp32.txt")).read().split("\n")
    digest = [l.split()[1] for l in text if l.startswith("csrc_sha256 ")]
    stages = {l.split()[1]: float(l.split()[2]) for l in text if l.startswith("stage ")}
    assert len(digest) == 1 and len(digest[0]) == 64
    assert set(stages) == {"fb", "weights", "gemm1", "gemm2", "bound"}
    assert all(v > 0 for v in stages.values())
    monkeypatch.setattr(bench, "csrc_digest", lambda: digest[0])
    assert bench.measured_traffic("fb", "paper_size_fp32") == stages["fb"]
    monkeypatch.setattr(bench, "csrc_digest", lambda: "0" * 64)
    assert bench.measured_traffic("fb", "paper_size_fp32") is None
    assert bench.measured_traffic("fb", "no_such_workload") is None
