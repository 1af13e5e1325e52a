"""GPU short-characteristics formal solution (the O(1)-per-pair method)
against the oracle's short-characteristics mode: J and Lambda* element by
element at 1e-12, shared-memory and global plane buffers, more directions
than one launch takes, converged solves, and the full 65^3 slab."""

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


def _lstar_close(L, Lo):
    scale = np.abs(Lo).reshape(27, -1).max(axis=0)
    return np.all(np.abs(L - Lo).reshape(27, -1).max(axis=0) <= 1e-12 * scale)


CASES = [
    dict(nx=17, ny=9, nz=6, seed=1),
    dict(nx=5, ny=5, nz=5, seed=2, chi_decades=6.0),
    dict(nx=3, ny=3, nz=4, seed=3),
    dict(nx=4, ny=3, nz=2, seed=4),
    dict(nx=13, ny=11, nz=7, seed=5, dx=0.7, dy=1.3, dz=0.9),
    dict(nx=12, ny=7, nz=9, seed=6, top_bc=W.BC_PLANCK, bottom_bc=W.BC_ZERO),
    dict(nx=10, ny=7, nz=6, seed=8, bottom_bc=W.BC_DIFFUSION),
    dict(nx=120, ny=110, nz=3, seed=9),     # two planes exceed the shared-memory budget
]


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("case", CASES, ids=lambda c: "{nx}x{ny}x{nz}".format(**c))
def test_sc_formal_solution_matches_oracle(R, oracle_mod, case, prec):
    kw = dict(case)
    p = W.random_slab(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), n_theta=6, n_phi=5,
                      seed=kw.pop("seed"), **kw)
    rng = np.random.default_rng(0)
    S = 0.5 + rng.random(p.B.shape) * 2.0
    precision = R.RT_DF64 if prec == "df64" else R.RT_FP64
    with R.Solver(p, precision=precision, fs_method=R.RT_FS_SHORT) as s:
        J, L = s.formal_solution(S)
        steps = R.rt_last_step_count(s.ctx)
    Jo, Lo = oracle_mod.formal_solution(p, S, method=oracle_mod.SHORT)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0), np.max(np.abs(J - Jo) / Jo)
    assert _lstar_close(L, Lo)
    assert steps == p.ndir * (p.nz - 1) * p.nx * p.ny


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_sc_more_directions_than_one_launch(R, oracle_mod, prec):
    """1100 directions: two launches of the march, their sums added in order."""
    p = W.random_slab(5, 4, 3, n_theta=44, n_phi=25, seed=10)
    assert p.ndir > 1024
    S = p.B * 1.3
    precision = R.RT_DF64 if prec == "df64" else R.RT_FP64
    with R.Solver(p, precision=precision, fs_method=R.RT_FS_SHORT) as s:
        J, L = s.formal_solution(S)
    Jo, Lo = oracle_mod.formal_solution(p, S, method=oracle_mod.SHORT)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0)
    assert _lstar_close(L, Lo)


def test_sc_switching_methods_and_errors(R, oracle_mod):
    p = W.random_slab(9, 8, 5, n_theta=4, n_phi=4, seed=11)
    S = p.B.copy()
    with R.Solver(p) as s:
        for m, om in ((R.RT_FS_SHORT, oracle_mod.SHORT), (R.RT_FS_LONG, oracle_mod.LONG),
                      (R.RT_FS_SHORT, oracle_mod.SHORT)):
            R.rt_set_fs_method(s.ctx, m)
            J, L = s.formal_solution(S)
            Jo, Lo = oracle_mod.formal_solution(p, S, method=om)
            assert np.allclose(J, Jo, rtol=RTOL, atol=0)
            assert _lstar_close(L, Lo)
        with pytest.raises(R.RtError):
            R.rt_set_fs_method(s.ctx, 2)
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        with pytest.raises(R.RtError):
            R.rt_set_fs_method(s.ctx, R.RT_FS_SHORT)
    with R.Solver(p, precision=R.RT_DF64, fs_method=R.RT_FS_SHORT) as s:
        with pytest.raises(R.RtError):
            R.rt_set_precision(s.ctx, R.RT_FP32_SWEEP)    # no FP32 short characteristics


@pytest.mark.parametrize("prec", ["fp64", "df64"])
@pytest.mark.parametrize("which", ["slab17", "random"])
def test_sc_converged_solve_matches_oracle(R, oracle_mod, which, prec):
    if which == "slab17":
        p = W.slab_small(n_theta=8, n_phi=8)
    else:
        p = W.random_slab(11, 10, 9, n_theta=6, n_phi=6, seed=51, eps_range=(1e-3, 1.0),
                          bottom_bc=W.BC_DIFFUSION)
    ro = oracle_mod.solve(p, tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12,
                          ng_period=4, fs_method=oracle_mod.SHORT)
    precision = R.RT_DF64 if prec == "df64" else R.RT_FP64
    with R.Solver(p, precision=precision, ng_period=4, fs_method=R.RT_FS_SHORT) as s:
        r = s.solve(tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12)
    assert r["converged"] and ro["converged"] and r["iters"] == ro["iters"]
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)


@pytest.mark.parametrize("prec", ["fp64", "df64"])
def test_sc_slab65_full_grid(R, oracle_mod, prec):
    """The 65^3 slab with 1024 directions, every voxel: J of one formal
    solution and its reproducibility."""
    p = W.slab_65()
    S = p.B.copy()
    precision = R.RT_DF64 if prec == "df64" else R.RT_FP64
    with R.Solver(p, precision=precision, fs_method=R.RT_FS_SHORT) as s:
        J1, _ = s.formal_solution(S, want_lstar=False)
        J2, _ = s.formal_solution(S, want_lstar=False)
    assert np.array_equal(J1, J2)
    Jo, _ = oracle_mod.formal_solution(p, S, lstar=False, method=oracle_mod.SHORT)
    assert np.allclose(J1, Jo, rtol=RTOL, atol=0), np.max(np.abs(J1 - Jo) / Jo)
