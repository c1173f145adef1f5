"""The C-ABI library builds for sm_103a, loads, exports every entry point
include/skei.h declares, and rejects bad arguments with SKEI_EINVAL before
touching a GPU (these run without a device)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
EINVAL = -1


@pytest.fixture(scope="module")
def lib():
    from paper_2411_05771_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def _declared():
    text = open(os.path.join(ROOT, "include", "skei.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(skei_[a-z0-9_]+)\s*\(", text)))


def test_header_declares_the_boundary():
    names = _declared()
    for required in ("skei_plan_create", "skei_proj_fwd", "skei_proj_adj", "skei_fbp",
                     "skei_fbp_adj", "skei_rotate", "skei_rotate_adj", "skei_ei_loss_fwd",
                     "skei_ei_loss_finish", "skei_ei_loss_bwd"):
        assert required in names


def test_every_declared_symbol_is_exported(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_built_for_sm_103a():
    from paper_2411_05771_gb300 import build
    assert "arch=compute_103a,code=sm_103a" in " ".join(build.ARCH)
    flags = open(os.path.join(os.path.dirname(build.LIB), "flags.txt")).read()
    assert "sm_103a" in flags


def test_validation_errors_need_no_gpu(lib):
    lib.skei_last_error.restype = ctypes.c_char_p
    lib.skei_plan_create.argtypes = [ctypes.c_int, ctypes.c_int, ctypes.c_int, ctypes.c_void_p,
                                     ctypes.POINTER(ctypes.c_void_p)]
    h = ctypes.c_void_p()
    assert lib.skei_plan_create(0, 0, 10, None, ctypes.byref(h)) == EINVAL
    assert b"N=0" in lib.skei_last_error()
    assert lib.skei_plan_create(64, 0, 0, None, ctypes.byref(h)) == EINVAL
    assert lib.skei_plan_create(64, -3, 10, None, ctypes.byref(h)) == EINVAL
    bad = (ctypes.c_double * 1)(float("nan"))
    assert lib.skei_plan_create(64, 0, 1, bad, ctypes.byref(h)) == EINVAL
    assert lib.skei_plan_create(64, 0, 1, None, None) == EINVAL

    vp = ctypes.c_void_p
    lib.skei_proj_fwd.argtypes = [vp, ctypes.c_int, vp, ctypes.c_int, vp, ctypes.c_int, vp, vp, vp]
    assert lib.skei_proj_fwd(None, 0, vp(16), 1, None, 1, None, vp(16), None) == EINVAL
    assert b"plan" in lib.skei_last_error()

    lib.skei_rotate.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.c_int, vp, ctypes.c_int,
                                vp, vp]
    # misaligned pointers, bad dtype, bad sizes
    assert lib.skei_rotate(0, vp(17), 1, 8, vp(32), 1, vp(64), None) == EINVAL
    assert b"aligned" in lib.skei_last_error()
    assert lib.skei_rotate(7, vp(16), 1, 8, vp(32), 1, vp(64), None) == EINVAL
    assert lib.skei_rotate(0, vp(16), 0, 8, vp(32), 1, vp(64), None) == EINVAL
    assert lib.skei_rotate(0, vp(16), 1, 8, vp(32), 0, vp(64), None) == EINVAL
    assert lib.skei_rotate(0, None, 1, 8, vp(32), 1, vp(64), None) == EINVAL

    lib.skei_fbp_workspace_size.restype = ctypes.c_size_t
    lib.skei_fbp_workspace_size.argtypes = [vp, ctypes.c_int, ctypes.c_int, ctypes.c_int]
    assert lib.skei_fbp_workspace_size(None, 0, 1, 1) == 0

    lib.skei_residual_add.argtypes = [ctypes.c_int, vp, vp, ctypes.c_int, ctypes.c_int64, vp, vp]
    assert lib.skei_residual_add(0, vp(16), vp(16), 0, 4, vp(16), None) == EINVAL
    assert lib.skei_version() >= 10000


def test_binding_rejects_host_tensors():
    torch = pytest.importorskip("torch")
    from paper_2411_05771_gb300 import skei as S
    with pytest.raises(TypeError):
        S.rotate(torch.zeros(1, 8, 8), torch.zeros(1, 1, dtype=torch.float64))


def test_batch_validation_needs_no_gpu(lib):
    vp = ctypes.c_void_p
    lib.skei_last_error.restype = ctypes.c_char_p
    lib.skei_batch_create.argtypes = [ctypes.c_int, vp, ctypes.c_int, ctypes.POINTER(vp)]
    lib.skei_batch_run.argtypes = [vp, vp]
    lib.skei_batch_tune.argtypes = [vp, ctypes.c_int, vp]
    lib.skei_batch_destroy.argtypes = [vp]
    h = vp()
    assert lib.skei_batch_create(0, vp(64), 1, None) == EINVAL
    assert lib.skei_batch_create(6, vp(64), 1, ctypes.byref(h)) == EINVAL
    assert b"operator" in lib.skei_last_error()
    assert lib.skei_batch_create(-1, vp(64), 1, ctypes.byref(h)) == EINVAL
    assert lib.skei_batch_create(0, None, 1, ctypes.byref(h)) == EINVAL
    assert lib.skei_batch_create(0, vp(64), 0, ctypes.byref(h)) == EINVAL
    assert not h.value
    assert lib.skei_batch_run(None, None) == EINVAL
    assert lib.skei_batch_tune(None, 3, None) == EINVAL
    assert lib.skei_batch_destroy(None) == 0


def test_check_entry_points_of_the_normal_build(lib):
    """The normal build is not the bounds-check build and reports no bits
    (without touching a GPU)."""
    assert lib.skei_check_build() == 0
    bits = ctypes.c_uint(7)
    assert lib.skei_check_status(ctypes.byref(bits), 1) == 0
    assert bits.value == 0


def test_every_call_is_an_nvtx_range(tmp_path):
    """Each C-ABI call opens and closes an NVTX range named after it (seen
    through a test injection library; calls rejected before any GPU work
    still do)."""
    import shutil
    import subprocess
    import sys
    from paper_2411_05771_gb300 import build
    gcc = shutil.which("gcc")
    if gcc is None:
        pytest.skip("no C compiler")
    probe = tmp_path / "libnvtx_probe.so"
    inc = os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(build.nvcc()))), "include")
    subprocess.run([gcc, "-shared", "-fPIC", "-O1", "-I", inc,
                    os.path.join(ROOT, "tests", "nvtx_probe.c"), "-o", str(probe)], check=True)
    log = tmp_path / "nvtx.log"
    code = (
        "import ctypes, sys\n"
        f"lib = ctypes.CDLL({build.build()!r})\n"
        "assert lib.skei_proj_fwd(None, 0, None, 1, None, 0, None, None, None) == -1\n"
        "assert lib.skei_rotate(0, None, 1, 0, None, 1, None, None) == -1\n")
    env = dict(os.environ, NVTX_INJECTION64_PATH=str(probe), SKEI_TEST_NVTX_LOG=str(log))
    subprocess.run([sys.executable, "-c", code], check=True, env=env)
    lines = log.read_text().split("\n")
    assert "push skei_proj_fwd" in lines and "push skei_rotate" in lines
    assert lines.count("pop") == sum(1 for x in lines if x.startswith("push "))
