"""The C-ABI library builds, loads and exports every symbol that
include/rt3d.h declares; without a GPU it fails loudly instead of falling
back to anything."""

import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for fn in os.listdir(os.path.join(ROOT, "include")):
        if fn.endswith(".h"):
            txt = open(os.path.join(ROOT, "include", fn)).read()
            txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
            names |= set(re.findall(r"\b(rt_[A-Za-z0-9_]+)\s*\(", txt))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1107_5719_gb300 import build as B
    path = B.build()
    from paper_1107_5719_gb300 import rt3d as R
    R.load(path)
    return path


def test_header_declares_the_boundary():
    names = _declared()
    for n in ["rt_create", "rt_destroy", "rt_set_grid", "rt_set_opacity", "rt_set_epsilon",
              "rt_set_planck", "rt_set_quadrature", "rt_set_boundary", "rt_formal_solution",
              "rt_os_step", "rt_solve", "rt_get_J", "rt_set_J"]:
        assert n in names, n


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", lib], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (rt_[A-Za-z0-9_]+)$", out, flags=re.M))
    missing = _declared() - exported
    assert not missing, f"declared but not exported: {sorted(missing)}"


def test_binding_covers_every_declared_symbol(lib):
    from paper_1107_5719_gb300 import rt3d as R
    assert _declared() == set(R.exported_names())
    for n in _declared():
        assert hasattr(R, n), n


def test_library_is_built_for_sm_103a(lib):
    from paper_1107_5719_gb300 import build as B
    assert B.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_checked_library_exports_the_same_symbols(lib):
    from paper_1107_5719_gb300 import build as B
    path = B.build(checked=True)
    out = subprocess.run(["nm", "-D", "--defined-only", path], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (rt_[A-Za-z0-9_]+)$", out, flags=re.M))
    assert not (_declared() - exported)


def test_no_gpu_fails_loudly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    from paper_1107_5719_gb300 import rt3d as R
    with pytest.raises(R.RtError):
        R.rt_create(0, R.RT_FP64)


def test_version_string(lib):
    from paper_1107_5719_gb300 import rt3d as R
    assert "rt3d" in R.rt_version()


def test_noalloc_rejects_bad_grids_before_touching_the_gpu(lib):
    """The allocation-free call checks its grid on the host first: these
    return RT_EINVAL without a CUDA call (the device pointers are never
    dereferenced), so they run without a GPU."""
    from paper_1107_5719_gb300 import rt3d as R, workloads as W
    mu, phi, w = W.quadrature(2, 2)
    fake = 1 << 20   # a device address that is never used
    for shape in [(2, 5, 5), (5, 5, 1), (5, 5, 65536)]:
        rc = R.rt_formal_solution_noalloc(*shape, 1.0, 1.0, 1.0, R.RT_BC_ZERO, R.RT_BC_PLANCK,
                                          mu, phi, w, fake, fake, fake, fake)
        assert rc == R.RT_EINVAL, shape
