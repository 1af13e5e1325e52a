"""The operator-splitting step as a CUDA graph (sweep loop in a WHILE node,
convergence test on the device) gives exactly the host-driven loop's
results: same sweep counts, bit-identical J, for Jacobi and Gauss-Seidel,
odd and even sweep limits, and whole solves."""

import numpy as np
import pytest

from paper_1107_5719_gb300 import workloads as W

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def R():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1107_5719_gb300 import build as B
    B.build()
    from paper_1107_5719_gb300 import rt3d
    rt3d.load()
    return rt3d


@pytest.mark.parametrize("method", [0, 1], ids=["jacobi", "gauss_seidel"])
@pytest.mark.parametrize("tol,max_sweeps", [(0.0, 7), (0.0, 8), (1e-12, 1000), (1e-6, 1000), (1e-9, 5)])
def test_os_step_graph_equals_host_loop(R, method, tol, max_sweeps):
    p = W.random_slab(13, 9, 8, n_theta=4, n_phi=4, seed=21, eps_range=(1e-3, 1.0))
    out = {}
    for graphs in (True, False):
        with R.Solver(p, os_method=method) as s:
            R.rt_set_graphs(s.ctx, graphs)
            Jfs, _ = s.formal_solution(p.B)
            out[graphs] = [s.os_step(Jfs, p.B, tol_inner=tol, max_sweeps=max_sweeps)
                           for _ in range(2)]       # the second call reuses the graph
    for (Jg, ng), (Jh, nh) in zip(out[True], out[False]):
        assert ng == nh
        assert np.array_equal(Jg, Jh)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
@pytest.mark.parametrize("method", [0, 1], ids=["jacobi", "gauss_seidel"])
def test_solve_graph_equals_host_loop(R, precision, method):
    p = W.random_slab(11, 10, 9, n_theta=6, n_phi=6, seed=51, eps_range=(1e-3, 1.0))
    prec = R.RT_FP64 if precision == "fp64" else R.RT_FP32_SWEEP
    tol = 1e-9 if precision == "fp64" else 5e-8
    res, stats = {}, {}
    for graphs in (True, False):
        with R.Solver(p, precision=prec, ng_period=4, ng_min_delta=1e-6, os_method=method) as s:
            R.rt_set_graphs(s.ctx, graphs)
            R.rt_reset_stats(s.ctx)
            res[graphs] = s.solve(tol=tol, max_iter=300, tol_inner=1e-11, max_sweeps=200)
            stats[graphs] = R.rt_get_stats(s.ctx)
    a, b = res[True], res[False]
    assert a["converged"] and a["iters"] == b["iters"]
    assert np.array_equal(a["sweeps"], b["sweeps"])
    assert np.array_equal(a["J"], b["J"])
    # with graphs, one host wait per outer iteration (Ng runs on the device)
    assert stats[True]["host_syncs"] == stats[True]["iterations"] == a["iters"]
    assert stats[False]["host_syncs"] > stats[True]["host_syncs"]


@pytest.mark.parametrize("precision", ["fp64", "df64"])
def test_all_options_together_match_oracle(R, oracle_mod, precision):
    """Short characteristics, red-black Gauss-Seidel, LTE-diffusion inner
    boundary, Planck outer boundary, Ng, the graph-driven sweeps and (for
    df64) the double-float arithmetic in one converged solve, against the
    oracle running the same options."""
    p = W.random_slab(10, 9, 8, n_theta=6, n_phi=5, seed=77, eps_range=(1e-3, 1.0),
                      top_bc=W.BC_PLANCK, bottom_bc=W.BC_DIFFUSION, dx=0.8, dz=1.2)
    ro = oracle_mod.solve(p, tol=1e-9, max_iter=300, tol_inner=0.0, max_sweeps=9, ng_period=4,
                          os_method=oracle_mod.GAUSS_SEIDEL, fs_method=oracle_mod.SHORT)
    prec = R.RT_FP64 if precision == "fp64" else R.RT_DF64
    with R.Solver(p, precision=prec, ng_period=4, fs_method=R.RT_FS_SHORT,
                  os_method=R.RT_OS_GAUSS_SEIDEL) as s:
        r = s.solve(tol=1e-9, max_iter=300, tol_inner=0.0, max_sweeps=9)
    assert r["converged"] and ro["converged"] and r["iters"] == ro["iters"]
    assert np.allclose(r["J"], ro["J"], rtol=1e-12, atol=0), np.max(np.abs(r["J"] - ro["J"]) / ro["J"])
