"""The bounds-checked build (librt3d_checked.so, RT3D_CHECKED=1): its guard
reports an out-of-range index as RT_EBOUNDS (exercised on an index that is
never dereferenced), it raises no false alarm on any formal-solution method,
precision or operator-splitting method, and its results match the normal
build's."""

import json
import os
import subprocess
import sys

import numpy as np
import pytest

pytestmark = pytest.mark.gpu
ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CHILD = r"""
import json, sys
import numpy as np
sys.path.insert(0, %(root)r)
from paper_1107_5719_gb300 import rt3d as R, workloads as W
R.load()
out = {"checked": R.rt_checked_build()}
p = W.random_slab(11, 9, 6, n_theta=6, n_phi=5, seed=3, bottom_bc=W.BC_DIFFUSION)
S = p.B * 1.2
res = {}
for name, kw in (("fp64", {}), ("fp32", dict(precision=R.RT_FP32_SWEEP)),
                 ("df64", dict(precision=R.RT_DF64)), ("short", dict(fs_method=R.RT_FS_SHORT))):
    with R.Solver(p, **kw) as s:
        J, L = s.formal_solution(S)
        res[name] = J.ravel().tolist()
p.src_order = 1
with R.Solver(p) as s:
    res["para"] = s.formal_solution(S)[0].ravel().tolist()
p.src_order = 0
for m in (R.RT_OS_JACOBI, R.RT_OS_GAUSS_SEIDEL):
    with R.Solver(p, ng_period=4, os_method=m) as s:
        r = s.solve(tol=1e-9, max_iter=200, tol_inner=1e-11, max_sweeps=300)
        res["solve%%d" %% m] = r["J"].ravel().tolist()
# an FP32-sweep solve through its finishing stage (double-float reference,
# then marches of the source change)
with R.Solver(p, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
    r = s.solve(tol=1e-9, max_iter=400)
    res["solve_fp32"] = r["J"].ravel().tolist()
with R.Solver(p) as s:
    rc1 = R.rt_bounds_selftest(s.ctx)
    msg = R.rt_last_error(s.ctx)
    rc2 = R.rt_bounds_selftest(s.ctx)
    J, _ = s.formal_solution(S)          # must succeed after the reports
out.update(res=res, rc1=rc1, rc2=rc2, msg=msg)
json.dump(out, open(sys.argv[1], "w"))
"""


def _run(tmp_path, checked):
    script = tmp_path / "child.py"
    script.write_text(CHILD % {"root": ROOT})
    out = tmp_path / ("checked.json" if checked else "plain.json")
    env = dict(os.environ, RT3D_CHECKED="1" if checked else "0")
    subprocess.run([sys.executable, str(script), str(out)], env=env, check=True, timeout=600)
    return json.load(open(out))


def test_checked_build_reports_and_matches(tmp_path):
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_5719_gb300 import build as B
    B.build_many((False, True))
    from paper_1107_5719_gb300 import rt3d as R
    plain = _run(tmp_path, False)
    chk = _run(tmp_path, True)
    assert chk["checked"] and not plain["checked"]
    assert plain["rc1"] == R.RT_OK and plain["rc2"] == R.RT_OK
    assert chk["rc1"] == R.RT_EBOUNDS and chk["rc2"] == R.RT_EBOUNDS
    assert "site 99" in chk["msg"]
    for k, v in plain["res"].items():
        a, b = np.array(v), np.array(chk["res"][k])
        # formal solutions agree to rounding; converged solves (delta < 1e-9)
        # to well within their tolerance; the FP32-sweep solve within its
        # march's rounding
        rtol = 1e-7 if k == "solve_fp32" else 1e-10 if k.startswith("solve") else 1e-13
        assert np.allclose(a, b, rtol=rtol, atol=0), (k, np.max(np.abs(a - b) / np.abs(a)))
