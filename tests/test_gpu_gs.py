"""GPU red-black Gauss-Seidel operator splitting (Sect. 2.3) against the
oracle: sweep by sweep, converged inner solves, whole outer iterations and
the batch path, element by element at 1e-12."""

import numpy as np
import pytest

from paper_1107_5719_gb300 import workloads as W

pytestmark = pytest.mark.gpu
RTOL = 1e-12


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


SHAPES = [(6, 4, 5, 1), (7, 5, 6, 2), (3, 3, 3, 3), (33, 9, 4, 4)]


@pytest.mark.parametrize("shape", SHAPES, ids=lambda s: "{}x{}x{}".format(*s[:3]))
def test_gs_os_step_matches_oracle(R, oracle_mod, shape):
    nx, ny, nz, seed = shape
    p = W.random_slab(nx, ny, nz, n_theta=4, n_phi=4, seed=seed, eps_range=(1e-3, 1.0))
    S = p.B.copy()
    Jfo, Lo = oracle_mod.formal_solution(p, S)
    # the first step of the outer iteration (J_old = B, S = B): an arbitrary
    # J_old can drive J_new through 0 in thick scattering voxels, where the
    # step amplifies J_fs - J_old by up to 1/eps
    Jold = p.B.copy()
    with R.Solver(p, os_method=R.RT_OS_GAUSS_SEIDEL) as s:
        Jfs, _ = s.formal_solution(S)
        for sweeps in (1, 2, 7):
            Jn, ns = s.os_step(Jfs, Jold, tol_inner=0.0, max_sweeps=sweeps)
            Jo, nso = oracle_mod.os_step(p, Lo, Jfo, Jold, tol_inner=0.0, max_sweeps=sweeps,
                                         method=oracle_mod.GAUSS_SEIDEL)
            assert ns == nso == sweeps
            assert np.allclose(Jn, Jo, rtol=RTOL, atol=0), np.max(np.abs(Jn - Jo) / Jo)
        Jn, ns = s.os_step(Jfs, Jold, tol_inner=1e-12, max_sweeps=1000)
        Jo, nso = oracle_mod.os_step(p, Lo, Jfo, Jold, tol_inner=1e-12, max_sweeps=1000,
                                     method=oracle_mod.GAUSS_SEIDEL)
        assert ns == nso
        assert np.allclose(Jn, Jo, rtol=RTOL, atol=0)


def test_gs_needs_fewer_sweeps_and_switching_methods(R, oracle_mod):
    p = W.random_slab(8, 7, 6, n_theta=4, n_phi=4, seed=9, eps_range=(1e-3, 1e-1))
    S = p.B.copy()
    Jfo, Lo = oracle_mod.formal_solution(p, S)
    Jold = p.B.copy()
    with R.Solver(p) as s:
        Jfs, _ = s.formal_solution(S)
        out = {}
        for m in (R.RT_OS_JACOBI, R.RT_OS_GAUSS_SEIDEL, R.RT_OS_JACOBI):
            R.rt_set_os_method(s.ctx, m)
            Jn, ns = s.os_step(Jfs, Jold, tol_inner=1e-12, max_sweeps=2000)
            Jo, nso = oracle_mod.os_step(p, Lo, Jfo, Jold, tol_inner=1e-12, max_sweeps=2000, method=m)
            assert ns == nso
            assert np.allclose(Jn, Jo, rtol=RTOL, atol=0)
            out.setdefault(m, ns)
        assert out[R.RT_OS_GAUSS_SEIDEL] < out[R.RT_OS_JACOBI]
        with pytest.raises(R.RtError):
            R.rt_set_os_method(s.ctx, 2)


@pytest.mark.parametrize("precision", ["fp64", "fp32"])
def test_gs_converged_solve_matches_oracle(R, oracle_mod, precision):
    p = W.random_slab(11, 10, 9, n_theta=6, n_phi=6, seed=51, eps_range=(1e-3, 1.0))
    if precision == "fp64":
        ro = oracle_mod.solve(p, tol=1e-8, max_iter=300, tol_inner=1e-10, max_sweeps=500,
                              ng_period=4, os_method=oracle_mod.GAUSS_SEIDEL)
        with R.Solver(p, ng_period=4, os_method=R.RT_OS_GAUSS_SEIDEL) as s:
            r = s.solve(tol=1e-8, max_iter=300, tol_inner=1e-10, max_sweeps=500)
        assert r["converged"] and r["iters"] == ro["iters"]
        assert np.array_equal(r["sweeps"], ro["sweeps"])
        assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)
    else:
        ro = oracle_mod.solve(p, tol=1e-11, max_iter=400, tol_inner=1e-12, max_sweeps=500)
        with R.Solver(p, precision=R.RT_FP32_SWEEP, os_method=R.RT_OS_GAUSS_SEIDEL) as s:
            r = s.solve(tol=5e-8, max_iter=400, tol_inner=1e-10, max_sweeps=500)
        assert r["converged"]
        assert np.allclose(r["J"], ro["J"], rtol=1e-6, atol=0)


def test_gs_batch_equals_single_solves(R):
    probs = [W.random_slab(9, 8, 7, n_theta=4, n_phi=4, seed=60 + i, eps_range=(1e-3, 1.0))
             for i in range(3)]
    b = R.rt_batch_create(probs, precision=R.RT_FP32_SWEEP)
    try:
        R.rt_batch_set_os_method(b, R.RT_OS_GAUSS_SEIDEL)
        r = R.rt_batch_solve(b, len(probs), tol=1e-6, max_iter=300, tol_inner=1e-10,
                             max_sweeps=300)
        assert r["converged"] and r["n_converged"] == len(probs)
        it = r["iters"]
        Jb = [R.rt_batch_get_J(b, i, (q.nz, q.ny, q.nx)) for i, q in enumerate(probs)]
    finally:
        R.rt_batch_destroy(b)
    for i, q in enumerate(probs):
        with R.Solver(q, precision=R.RT_FP32_SWEEP, os_method=R.RT_OS_GAUSS_SEIDEL) as s:
            r = s.solve(tol=1e-6, max_iter=300, tol_inner=1e-10, max_sweeps=300)
        assert r["iters"] == it[i]
        assert np.array_equal(r["J"], Jb[i])
