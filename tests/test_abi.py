"""The C-ABI library without a GPU: it loads, exports every entry point that
include/gsicp.h declares, and rejects bad arguments before touching a device."""
import ctypes as C
import os
import re
import subprocess
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "gsicp.h")


@pytest.fixture(scope="module")
def lib():
    from paper_2403_12550_b300.build import build
    return C.CDLL(build())


def declared_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(gsicp_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_path(lib):
    names = declared_functions()
    for required in ("gsicp_build_map_index", "gsicp_source_covariances", "gsicp_register",
                     "gsicp_depth_to_points", "gsicp_track_frame"):
        assert required in names
    assert len(names) >= 15


def test_every_declared_symbol_is_exported(lib):
    for name in declared_functions():
        assert hasattr(lib, name), name


def test_invalid_arguments_are_rejected_without_a_device(lib):
    INVALID = 1
    lib.gsicp_ctx_create.argtypes = [C.c_void_p]
    assert lib.gsicp_ctx_create(None) == INVALID
    lib.gsicp_register.argtypes = [C.c_void_p] * 5 + [C.c_void_p] * 9
    lib.gsicp_register.restype = C.c_int
    assert lib.gsicp_register(*([None] * 14)) == INVALID
    lib.gsicp_build_map_index.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                          C.c_void_p]
    assert lib.gsicp_build_map_index(None, None, None, 0, None, None, None) == INVALID
    lib.gsicp_source_covariances.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int64, C.c_void_p, C.c_void_p,
                                             C.c_void_p, C.c_void_p]
    assert lib.gsicp_source_covariances(None, None, None, 10, None, None, None, None) == INVALID
    lib.gsicp_frame_covariances.argtypes = [C.c_void_p] * 2 + [C.c_int] * 2 + [C.c_void_p, C.c_int, C.c_float,
                                                                               C.c_float] + [C.c_void_p] * 4 + \
        [C.c_int64, C.c_void_p, C.c_void_p]
    assert lib.gsicp_frame_covariances(None, None, 8, 8, None, 1, 0.1, 10.0, None, None, None, None, 64, None,
                                       None) == INVALID
    lib.gsicp_ctx_frame_stats.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.gsicp_ctx_frame_stats(None, None) == INVALID
    lib.gsicp_register_batch.argtypes = [C.c_void_p, C.c_int] + [C.c_void_p] * 12
    assert lib.gsicp_register_batch(None, 2, *([None] * 12)) == INVALID
    lib.gsicp_selftest_batch_timeout.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.gsicp_selftest_batch_timeout(None, None) == INVALID
    lib.gsicp_tracker_create.argtypes = [C.c_void_p, C.c_int, C.c_float, C.c_float] + [C.c_void_p] * 4
    assert lib.gsicp_tracker_create(None, 2, 0.1, 10.0, None, None, None, None) == INVALID
    lib.gsicp_tracker_frame.argtypes = [C.c_void_p, C.c_void_p, C.c_int, C.c_int] + [C.c_void_p] * 5
    assert lib.gsicp_tracker_frame(None, None, 8, 8, None, None, None, None, None) == INVALID
    lib.gsicp_tracker_destroy(None)
    lib.gsicp_ctx_last_residual.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    assert lib.gsicp_ctx_last_residual(None, None, None) == INVALID
    lib.gsicp_ctx_set_coop_walks.argtypes = [C.c_void_p, C.c_int]
    assert lib.gsicp_ctx_set_coop_walks(None, 4) == INVALID
    lib.gsicp_surrogate_create.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.gsicp_surrogate_create(None, None) == INVALID
    lib.gsicp_surrogate_destroy(None)
    lib.gsicp_surrogate_set_timing.argtypes = [C.c_void_p, C.c_int]
    assert lib.gsicp_surrogate_set_timing(None, 1) == INVALID
    lib.gsicp_surrogate_layer_times.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.gsicp_surrogate_layer_times(None, None) == INVALID
    lib.gsicp_surrogate_get_weights.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.gsicp_surrogate_get_weights(None, None) == INVALID
    lib.gsicp_surrogate_set_weights.argtypes = [C.c_void_p, C.c_void_p]
    assert lib.gsicp_surrogate_set_weights(None, None) == INVALID
    lib.gsicp_surrogate_covariances.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                                C.c_int, C.c_float, C.c_float] + [C.c_void_p] * 5 + \
        [C.c_int64, C.c_void_p, C.c_void_p]
    assert lib.gsicp_surrogate_covariances(None, None, None, 8, 8, None, 1, 0.1, 10.0, None, None, None, None, None,
                                           64, None, None) == INVALID
    lib.gsicp_surrogate_train_step.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_int, C.c_int, C.c_void_p,
                                               C.c_int, C.c_float, C.c_float, C.c_void_p, C.c_void_p, C.c_float,
                                               C.c_int] + [C.c_void_p] * 4
    assert lib.gsicp_surrogate_train_step(None, None, None, 8, 8, None, 1, 0.1, 10.0, None, None, 1e-3, 1,
                                          None, None, None, None) == INVALID
    lib.gsicp_track_frame_surrogate.argtypes = [C.c_void_p] * 3 + [C.c_int, C.c_int, C.c_void_p, C.c_int,
                                                                   C.c_float, C.c_float] + [C.c_void_p] * 11
    assert lib.gsicp_track_frame_surrogate(None, None, None, 8, 8, None, 1, 0.1, 10.0, *([None] * 11)) == INVALID
    lib.gsicp_tracker_set_surrogate.argtypes = [C.c_void_p, C.c_void_p, C.c_float, C.c_int, C.c_int]
    assert lib.gsicp_tracker_set_surrogate(None, None, 1.1, 30, 1) == INVALID
    lib.gsicp_map_size.restype = C.c_int64
    assert lib.gsicp_map_size(None) == 0
    lib.gsicp_map_destroy(None)
    lib.gsicp_ctx_destroy(None)
    lib.gsicp_status_string.restype = C.c_char_p
    assert b"degenerate" in lib.gsicp_status_string(4)
    lib.gsicp_version.restype = C.c_char_p
    assert lib.gsicp_version().startswith(b"0.")


def test_package_fails_loudly_without_the_library(tmp_path):
    """With no libgsicp.so next to it the binding refuses to import: there is no fallback."""
    import shutil
    pkg = os.path.join(ROOT, "paper_2403_12550_b300")
    dst = tmp_path / "paper_2403_12550_b300"
    shutil.copytree(pkg, dst, ignore=shutil.ignore_patterns("*.so", "__pycache__"))
    r = subprocess.run([sys.executable, "-c", "import paper_2403_12550_b300"], cwd=tmp_path,
                       capture_output=True, text=True)
    assert r.returncode != 0 and "libgsicp.so is missing" in r.stderr


def test_product_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2403_12550_b300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "oracle" not in text.lower(), f


def test_binding_rejects_host_or_mistyped_tensors_before_the_call():
    # the binding hands the library device pointers only: a host tensor, another dtype, a strided
    # view or a wrong row width is refused in Python, before any C call
    import torch
    import paper_2403_12550_b300 as g
    for bad in (torch.zeros(4, 3), torch.zeros(4, 3, dtype=torch.float64), torch.zeros(3, 4).t()):
        with pytest.raises(TypeError):
            g._dev(bad, cols=3)
    assert g._dev(None) is None
    pose = g._pose(np.arange(16.0).reshape(4, 4))
    assert list(pose) == list(np.arange(16.0))
    with pytest.raises(g.GsicpError) as e:
        g._check(g.ERR_INVALID_ARG, "somewhere")
    assert "somewhere" in str(e.value)
    assert g._check(g.ERR_DEGENERATE, "x", allow=(g.ERR_DEGENERATE,)) == g.ERR_DEGENERATE


def _kernel_body_start(src: str, name: str) -> str:
    """The first statement of __global__ kernel `name` in src (templates included)."""
    m = re.search(r"__global__\s+void\s+(?:__launch_bounds__\((?:[^()]|\([^()]*\))*\)\s+)?" + re.escape(name) + r"\s*\(",
                  src)
    assert m, name
    depth, i = 0, m.end() - 1
    while True:  # the parameter list, then the body's opening brace
        c = src[i]
        depth += c == "("
        depth -= c == ")"
        i += 1
        if depth == 0:
            break
    body = src[src.index("{", i) + 1:]
    return body.lstrip().split(";", 1)[0]


def test_dependent_launches_wait_for_the_kernel_before_them():
    """A kernel launched as a programmatic dependent may start before the kernel ahead of it in the
    stream has finished; every such kernel must wait (griddepcontrol.wait) before it reads
    anything.  Checks each launch_dependent target and the Gauss-Newton iteration kernel."""
    csrc = os.path.join(ROOT, "paper_2403_12550_b300", "csrc")
    src = "".join(open(os.path.join(csrc, f)).read() for f in sorted(os.listdir(csrc)) if f.endswith((".cu", ".cuh")))
    targets = sorted(set(re.findall(r"launch_dependent\(\s*([a-z_0-9]+)", src)) - {"void"})
    assert len(targets) >= 14, targets
    for name in targets:
        assert _kernel_body_start(src, name) == "wait_prior_grid()", name
    assert "griddepcontrol.wait" in _kernel_body_start(src, "gicp_iter_kernel")
