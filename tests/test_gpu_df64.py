"""GPU double-float ("RT_DF64") form: the march in pairs of FP32 numbers on
the FP32 pipes, FP64 J, Lambda*, operator splitting and convergence.  It is
held to the FP64 path's bar: J within 1e-12 of the FP64 oracle, element by
element, for single formal solutions and converged solves."""

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


CASES = [
    dict(nx=17, ny=9, nz=6, seed=1),
    dict(nx=5, ny=5, nz=5, seed=2, chi_decades=6.0),
    dict(nx=3, ny=3, nz=4, seed=3),
    dict(nx=4, ny=3, nz=2, seed=4),
    dict(nx=13, ny=11, nz=7, seed=5, dx=0.7, dy=1.3, dz=0.9),
    dict(nx=12, ny=7, nz=9, seed=6, top_bc=W.BC_PLANCK, bottom_bc=W.BC_ZERO),
    dict(nx=10, ny=7, nz=6, seed=8, bottom_bc=W.BC_DIFFUSION),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "{nx}x{ny}x{nz}".format(**c))
def test_df64_formal_solution_matches_oracle(R, oracle_mod, case):
    kw = dict(case)
    p = W.random_slab(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), n_theta=6, n_phi=5,
                      seed=kw.pop("seed"), **kw)
    rng = np.random.default_rng(0)
    S = 0.5 + rng.random(p.B.shape) * 2.0
    with R.Solver(p, precision=R.RT_DF64) as s:
        J, L = s.formal_solution(S)
    Jo, Lo = oracle_mod.formal_solution(p, S)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0), np.max(np.abs(J - Jo) / Jo)
    scale = np.abs(Lo).reshape(27, -1).max(axis=0)
    assert np.all(np.abs(L - Lo).reshape(27, -1).max(axis=0) <= 1e-12 * scale)


def test_df64_slab65_sampled(R, oracle_mod):
    p = W.slab_65()
    S = p.eps * p.B + (1 - p.eps) * p.B
    with R.Solver(p, precision=R.RT_DF64) as s:
        J, _ = s.formal_solution(want_lstar=False)
    rng = np.random.default_rng(5)
    ks = np.concatenate([np.arange(p.nz), rng.integers(0, p.nz, 63)])
    vox = ks * p.nx * p.ny + rng.integers(0, p.nx * p.ny, ks.shape[0])
    Jo = oracle_mod.mean_intensity_at(p, S, vox)
    assert np.allclose(J.ravel()[vox], Jo, rtol=RTOL, atol=0), np.max(np.abs(J.ravel()[vox] - Jo) / Jo)


@pytest.mark.parametrize("which", ["slab17", "random"])
def test_df64_converged_solve_matches_oracle(R, oracle_mod, which):
    if which == "slab17":
        p = W.slab_small(n_theta=8, n_phi=8)
    else:
        p = W.random_slab(11, 10, 9, n_theta=6, n_phi=6, seed=51, eps_range=(1e-3, 1.0))
    ro = oracle_mod.solve(p, tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12, ng_period=4)
    with R.Solver(p, precision=R.RT_DF64, ng_period=4) as s:
        r = s.solve(tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12)
    assert r["converged"] and ro["converged"] and r["iters"] == ro["iters"]
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0), np.max(np.abs(r["J"] - ro["J"]) / ro["J"])


def test_df64_deterministic(R):
    p = W.random_slab(19, 8, 7, n_theta=8, n_phi=6, seed=12)
    out = []
    for groups in (0, 1, 8):
        with R.Solver(p, precision=R.RT_DF64, groups=groups) as s:
            out.append(s.formal_solution(want_lstar=False)[0])
    for J in out[1:]:
        assert np.array_equal(J, out[0])
