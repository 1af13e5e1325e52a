"""GPU FP64 path against the FP64 oracle, element by element.

Formal solution J and Lambda* (Sect. 2.2), the operator-splitting step
(Sect. 2.3) and the converged outer iteration (Sect. 2) on slabs that span
several 128-voxel tiles with a ragged tail, edge cases (nz = 2, 3x3
planes that alias the neighbourhood, vertical and grazing rays, both
boundary modes) and the 65^3, 32x32-direction slab on sampled voxels.
Tolerance: 1e-12 relative in J (FP64 path).
"""

import math

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


def _lstar_close(L, Lo, rtol=RTOL):
    scale = np.abs(Lo).reshape(27, -1).max(axis=0)        # per voxel
    err = np.abs(L - Lo).reshape(27, -1).max(axis=0)
    return bool(np.all(err <= rtol * np.maximum(scale, 1e-300)))


CASES = [
    dict(nx=17, ny=9, nz=6, seed=1),                      # 153-voxel planes: 2 tiles, ragged
    dict(nx=5, ny=5, nz=5, seed=2),
    dict(nx=3, ny=3, nz=4, seed=3),                        # smallest periodic plane
    dict(nx=4, ny=3, nz=2, seed=4),                        # nz = 2
    dict(nx=13, ny=11, nz=7, seed=5, dx=0.7, dy=1.3, dz=0.9),
    dict(nx=12, ny=7, nz=9, seed=6, top_bc=W.BC_PLANCK, bottom_bc=W.BC_ZERO),
    dict(nx=6, ny=6, nz=8, seed=7, top_bc=W.BC_ZERO, bottom_bc=W.BC_ZERO, chi_decades=6.0),
    dict(nx=10, ny=7, nz=6, seed=8, bottom_bc=W.BC_DIFFUSION),      # LTE-diffusion inner boundary
    dict(nx=5, ny=4, nz=2, seed=9, top_bc=W.BC_PLANCK, bottom_bc=W.BC_DIFFUSION, dz=0.6),
]


@pytest.mark.parametrize("case", CASES, ids=lambda c: "{nx}x{ny}x{nz}".format(**c))
def test_formal_solution_and_lstar_match_oracle(R, oracle_mod, case):
    kw = dict(case)
    p = W.random_slab(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), n_theta=6, n_phi=5,
                      seed=kw.pop("seed"), **kw)
    rng = np.random.default_rng(0)
    S = 0.5 + rng.random(p.B.shape) * 2.0
    with R.Solver(p) as s:
        J, L = s.formal_solution(S)
        steps = R.rt_last_step_count(s.ctx)
    Jo, Lo = oracle_mod.formal_solution(p, S)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0)
    assert _lstar_close(L, Lo)
    assert steps > 0


def test_slab17_formal_solution_and_lstar(R, oracle_mod):
    p = W.slab_small()
    S = p.eps * p.B + (1 - p.eps) * p.B
    with R.Solver(p) as s:
        J, L = s.formal_solution()        # S from the iterate J = B
    Jo, Lo = oracle_mod.formal_solution(p, S)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0)
    assert _lstar_close(L, Lo)


def test_cutoff_does_not_change_j(R):
    p = W.slab_small(n_theta=8, n_phi=8)
    with R.Solver(p, cutoff=0.0) as s:
        J0, _ = s.formal_solution()
        n0 = R.rt_last_step_count(s.ctx)
    with R.Solver(p) as s:
        J1, _ = s.formal_solution()
        n1 = R.rt_last_step_count(s.ctx)
    assert n1 < n0
    assert np.allclose(J1, J0, rtol=1e-15, atol=0)


def test_deterministic_and_independent_of_launch_shape(R):
    p = W.random_slab(19, 8, 7, n_theta=8, n_phi=6, seed=12)
    Js = []
    for groups in (0, 1, 2, 4, 8, 0):
        with R.Solver(p, groups=groups) as s:
            Js.append(s.formal_solution(want_lstar=False)[0])
    for J in Js[1:]:
        assert np.array_equal(J, Js[0])


def test_special_directions(R, oracle_mod):
    """Vertical rays (mu = +-1), grazing rays and exact-lattice 45-degree rays."""
    nx, ny, nz = 7, 5, 6
    mu = np.array([1.0, -1.0, 1e-3, -1e-3, 1 / math.sqrt(2), -1 / math.sqrt(2)])
    phi = np.array([0.3, 1.1, 0.7, 4.0, 0.0, math.pi])
    w = np.full(6, 1 / 6)
    base = W.random_slab(nx, ny, nz, seed=31)
    p = W.Problem(nx, ny, nz, base.chi, base.eps, base.B, mu, phi, w)
    S = base.B * 1.3
    with R.Solver(p) as s:
        J, L = s.formal_solution(S)
    Jo, Lo = oracle_mod.formal_solution(p, S)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0)
    assert _lstar_close(L, Lo)


def test_os_step_matches_oracle(R, oracle_mod):
    p = W.random_slab(17, 9, 6, n_theta=4, n_phi=6, seed=41, eps_range=(1e-4, 1.0))
    S = p.eps * p.B + (1 - p.eps) * p.B
    rng = np.random.default_rng(3)
    Jold = p.B * (0.3 + rng.random(p.B.shape))
    with R.Solver(p) as s:
        Jfs, L = s.formal_solution(S)
        Jn, ns = s.os_step(Jfs, Jold, tol_inner=0.0, max_sweeps=25)
        Jn2, ns2 = s.os_step(Jfs, Jold, tol_inner=1e-12, max_sweeps=1000)
    Jfo, Lo = oracle_mod.formal_solution(p, S)
    Jno, _ = oracle_mod.os_step(p, Lo, Jfo, Jold, tol_inner=0.0, max_sweeps=25)
    assert ns == 25
    assert np.allclose(Jn, Jno, rtol=RTOL, atol=0)
    Jno2, nso2 = oracle_mod.os_step(p, Lo, Jfo, Jold, tol_inner=1e-12, max_sweeps=1000)
    assert ns2 == nso2
    assert np.allclose(Jn2, Jno2, rtol=RTOL, atol=0)


@pytest.mark.parametrize("which", ["slab17", "random"])
def test_converged_solve_matches_oracle(R, oracle_mod, which):
    """Same iteration from J = B with a fixed inner sweep count: the
    iteration counts agree and so does the converged J."""
    if which == "slab17":
        p = W.slab_small(n_theta=8, n_phi=8)
    else:
        p = W.random_slab(11, 10, 9, n_theta=6, n_phi=6, seed=51, eps_range=(1e-3, 1.0))
    ro = oracle_mod.solve(p, tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12)
    assert ro["converged"]
    with R.Solver(p) as s:
        r = s.solve(tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12)
    assert r["converged"]
    assert r["iters"] == ro["iters"]
    assert np.allclose(r["deltas"], ro["deltas"], rtol=1e-6, atol=1e-300)
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)


@pytest.mark.parametrize("period,min_delta", [(4, 0.0), (5, 0.0), (4, 1e-5)])
def test_ng_accelerated_solve_matches_oracle(R, oracle_mod, period, min_delta):
    """Ng-accelerated outer iteration: same iteration count and J as the
    oracle's Ng-accelerated iteration, and fewer iterations than plain."""
    p = W.slab_small(n_theta=8, n_phi=8)
    ro = oracle_mod.solve(p, tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12,
                          ng_period=period, ng_min_delta=min_delta)
    with R.Solver(p, ng_period=period, ng_min_delta=min_delta) as s:
        r = s.solve(tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12)
    assert r["converged"] and ro["converged"]
    assert r["iters"] == ro["iters"]
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)
    with R.Solver(p) as s:
        plain = s.solve(tol=1e-8, max_iter=300, tol_inner=0.0, max_sweeps=12)
    assert r["iters"] < plain["iters"]


def test_converged_solve_tolerance_driven_inner(R, oracle_mod):
    p = W.slab_small(n_theta=8, n_phi=8)
    ro = oracle_mod.solve(p, tol=1e-8, max_iter=300)
    with R.Solver(p) as s:
        r = s.solve(tol=1e-8, max_iter=300)
    assert r["converged"] and r["iters"] == ro["iters"]
    assert np.array_equal(r["sweeps"], ro["sweeps"])
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)


def test_converged_solve_with_diffusion_boundary(R, oracle_mod):
    p = W.random_slab(9, 8, 10, n_theta=6, n_phi=4, seed=55, eps_range=(1e-3, 1.0),
                      bottom_bc=W.BC_DIFFUSION)
    ro = oracle_mod.solve(p, tol=1e-9, max_iter=400, tol_inner=0.0, max_sweeps=12)
    with R.Solver(p) as s:
        r = s.solve(tol=1e-9, max_iter=400, tol_inner=0.0, max_sweeps=12)
    assert r["converged"] and ro["converged"] and r["iters"] == ro["iters"]
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)


def test_diffusion_boundary_rejected_at_the_top(R):
    ctx = R.rt_create(0, R.RT_FP64)
    try:
        with pytest.raises(R.RtError) as e:
            R.rt_set_boundary(ctx, R.RT_BC_DIFFUSION, R.RT_BC_PLANCK)
        assert e.value.code == R.RT_EINVAL
    finally:
        R.rt_destroy(ctx)


def test_pure_absorption_limit(R, oracle_mod):
    """eps = 1: J_new = J_fs, the solve converges on the second pass."""
    p = W.random_slab(9, 9, 5, seed=61, eps_range=(1.0, 1.0))
    with R.Solver(p) as s:
        r = s.solve(tol=1e-14, max_iter=10)
    ro = oracle_mod.solve(p, tol=1e-14, max_iter=10)
    assert r["converged"] and r["iters"] == ro["iters"] == 2
    assert np.allclose(r["J"], ro["J"], rtol=RTOL, atol=0)


def test_checkpoint_resume(R):
    p = W.random_slab(9, 8, 7, n_theta=4, n_phi=4, seed=71, eps_range=(1e-2, 1.0))
    with R.Solver(p) as s:
        full = s.solve(tol=0.0, max_iter=8, tol_inner=0.0, max_sweeps=10)
    with R.Solver(p) as s:
        s.solve(tol=0.0, max_iter=3, tol_inner=0.0, max_sweeps=10)
        Jmid = R.rt_get_J(s.ctx, s.shape)
    with R.Solver(p) as s:
        R.rt_set_J(s.ctx, Jmid)
        rest = s.solve(tol=0.0, max_iter=5, tol_inner=0.0, max_sweeps=10)
    assert np.array_equal(rest["J"], full["J"])


def test_slab65_sampled_formal_solution(R, oracle_mod):
    """65^3 slab, 32 x 32 directions, the launch the benchmark times: J and
    the 27 Lambda* entries at 160 sampled voxels (every depth plus random
    ones) against the oracle at the FP64 bar."""
    p = W.slab_65()
    S = p.eps * p.B + (1 - p.eps) * p.B
    with R.Solver(p) as s:
        J, L = s.formal_solution()
    rng = np.random.default_rng(5)
    ks = np.concatenate([np.arange(p.nz), rng.integers(0, p.nz, 95)])
    vox = ks * p.nx * p.ny + rng.integers(0, p.nx * p.ny, ks.shape[0])
    Jo = oracle_mod.mean_intensity_at(p, S, vox)
    assert np.allclose(J.ravel()[vox], Jo, rtol=RTOL, atol=0)
    Lo = oracle_mod.lstar_at(p, vox)                      # [160][27]
    Lg = L.reshape(27, -1)[:, vox].T
    scale = np.abs(Lo).max(axis=1, keepdims=True)
    assert np.all(np.abs(Lg - Lo) <= RTOL * scale), np.max(np.abs(Lg - Lo) / scale)
    assert np.all(L >= 0)
    assert np.all(L.sum(axis=0) <= 1.0 + 1e-12)


def test_slab65_converged_fixed_point(R, oracle_mod):
    """Converged 65^3 solve (FP64, outer tolerance 1e-11; the iterate's
    delta stops falling near 3e-12, its rounding floor): J is the fixed
    point J = J_fs(eps B + (1-eps) J) of the oracle's formal solution at 160
    sampled voxels to 1e-10 relative."""
    p = W.slab_65()
    with R.Solver(p, ng_period=4) as s:
        r = s.solve(tol=1e-11, max_iter=400, tol_inner=1e-14, max_sweeps=4000)
    assert r["converged"]
    J = r["J"]
    S = p.eps * p.B + (1 - p.eps) * J
    rng = np.random.default_rng(8)
    ks = np.concatenate([np.arange(p.nz), rng.integers(0, p.nz, 95)])
    vox = ks * p.nx * p.ny + rng.integers(0, p.nx * p.ny, ks.shape[0])
    Jo = oracle_mod.mean_intensity_at(p, S, vox)
    rel = np.abs(Jo - J.ravel()[vox]) / J.ravel()[vox]
    assert rel.max() < 1e-10, rel.max()


@pytest.mark.parametrize("bad", ["chi0", "chi_nan", "eps0", "eps_big", "mu0", "wsum", "grid"])
def test_invalid_inputs_rejected(R, bad):
    p = W.random_slab(5, 4, 3, seed=81)
    ctx = R.rt_create(0, R.RT_FP64)
    try:
        if bad == "grid":
            for shape in [(2, 5, 5), (5, 5, 1), (5, 5, 65536)]:
                with pytest.raises(R.RtError) as e:
                    R.rt_set_grid(ctx, *shape)
                assert e.value.code == R.RT_EINVAL
            return
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz)
        chi, eps, mu, w = p.chi.copy(), p.eps.copy(), p.mu.copy(), p.w.copy()
        if bad == "chi0":
            chi[1, 2, 3] = 0.0
        if bad == "chi_nan":
            chi[0, 0, 0] = np.nan
        if bad == "eps0":
            eps[2, 1, 0] = 0.0
        if bad == "eps_big":
            eps[0, 1, 1] = 1.5
        if bad == "mu0":
            mu[3] = 0.0
        if bad == "wsum":
            w = w * 1.01
        with pytest.raises(R.RtError) as e:
            R.rt_set_quadrature(ctx, mu, p.phi, w)
            R.rt_set_opacity(ctx, chi)
            R.rt_set_epsilon(ctx, eps)
        assert e.value.code == R.RT_EINVAL
    finally:
        R.rt_destroy(ctx)


def test_state_errors(R):
    ctx = R.rt_create(0, R.RT_FP64)
    try:
        with pytest.raises(R.RtError) as e:
            R.rt_formal_solution(ctx, None, (3, 3, 3))
        assert e.value.code == R.RT_ESTATE
    finally:
        R.rt_destroy(ctx)


def test_device_pointer_calls(R, oracle_mod):
    import torch
    p = W.random_slab(10, 9, 6, n_theta=4, n_phi=4, seed=91)
    dev = torch.device("cuda:0")
    chi = torch.from_numpy(p.chi).to(dev)
    eps = torch.from_numpy(p.eps).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    S = torch.from_numpy(p.B * 0.8).to(dev)
    Jfs = torch.empty_like(B)
    L = torch.empty((27, *p.B.shape), dtype=torch.float64, device=dev)
    ctx = R.rt_create(0, R.RT_FP64)
    try:
        R.rt_set_stream(ctx, torch.cuda.current_stream())
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz)
        R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
        R.rt_set_opacity_dev(ctx, chi)
        R.rt_set_epsilon_dev(ctx, eps)
        R.rt_set_planck_dev(ctx, B)
        R.rt_formal_solution_dev(ctx, S, Jfs, L)
        torch.cuda.synchronize()
        Jo, Lo = oracle_mod.formal_solution(p, p.B * 0.8)
        assert np.allclose(Jfs.cpu().numpy(), Jo, rtol=RTOL, atol=0)
        assert _lstar_close(L.cpu().numpy(), Lo)
        Jn = torch.empty_like(B)
        R.rt_os_step_dev(ctx, Jfs, B, Jn, 0.0, 7)
        Jno, _ = oracle_mod.os_step(p, Lo, Jo, p.B, tol_inner=0.0, max_sweeps=7)
        assert np.allclose(Jn.cpu().numpy(), Jno, rtol=RTOL, atol=0)
        Jout = torch.empty_like(B)
        it, delta, conv = R.rt_solve_dev(ctx, Jout, tol=1e-10, max_iter=100)
        ro = oracle_mod.solve(p, tol=1e-10, max_iter=100)
        assert conv and it == ro["iters"]
        assert np.allclose(Jout.cpu().numpy(), ro["J"], rtol=RTOL, atol=0)
    finally:
        R.rt_destroy(ctx)


def _weights_mp(x):
    import mpmath
    mpmath.mp.dps = 40
    x = mpmath.mpf(x)
    e = mpmath.exp(-x)
    q = -mpmath.expm1(-x) / x
    return float(1 - q), float(q - e), float(e)


@pytest.mark.parametrize("precision,rtol", [(0, 4e-15), (1, 2e-6)])
def test_device_segment_weights_against_high_precision(R, precision, rtol):
    """The march's own segment weights and exp(-x) on the GPU against a
    40-digit evaluation of their definition (mpmath)."""
    pytest.importorskip("mpmath")
    import torch
    xs = np.concatenate([np.logspace(-10, np.log10(690.0), 400),
                         [0.25 * (1 - 1e-15), 0.25, 0.75 * (1 - 1e-7), 0.75, 1.0, 2.0, 50.0]])
    dev = torch.device("cuda:0")
    x = torch.from_numpy(xs).to(dev)
    wc, wu, e = torch.empty_like(x), torch.empty_like(x), torch.empty_like(x)
    assert R.rt_segment_weights(precision, x, wc, wu, e) == 0
    torch.cuda.synchronize()
    wc, wu, e = wc.cpu().numpy(), wu.cpu().numpy(), e.cpu().numpy()
    for i, xv in enumerate(xs):
        if precision == 1:
            xv = float(np.float32(xv))
        rc, ru, re = _weights_mp(xv)
        assert abs(wc[i] - rc) <= rtol * rc, (xv, wc[i], rc)
        assert abs(wu[i] - ru) <= rtol * ru, (xv, wu[i], ru)
        # FP32: rounding x*log2(e) to FP32 costs ~x*6e-8 of relative accuracy in e
        etol = rtol * re if precision == 0 else 1.5e-7 * (1.0 + xv) * re + 1e-37
        assert abs(e[i] - re) <= etol, (xv, e[i], re)


def test_not_converged_is_reported_and_outputs_stay_valid(R, oracle_mod):
    """max_iter reached before tol: the C call returns RT_ENOTCONV, J and the
    per-iteration deltas are still those of the iterations run."""
    import ctypes as C
    p = W.random_slab(7, 6, 5, n_theta=4, n_phi=4, seed=93, eps_range=(1e-3, 1e-2))
    with R.Solver(p) as s:
        lib = R.load()
        J = np.empty(s.shape)
        it, last = C.c_int(), C.c_double()
        d = np.zeros(3)
        rc = lib.rt_solve(s.ctx, 1e-12, 3, 0.0, 10, J.ctypes.data, C.byref(it), C.byref(last),
                          d.ctypes.data, None)
        assert rc == R.RT_ENOTCONV and it.value == 3 and last.value == d[-1] > 0
        assert "not converged" in R.rt_last_error(s.ctx)
    ro = oracle_mod.solve(p, tol=0.0, max_iter=3, tol_inner=0.0, max_sweeps=10)
    assert np.allclose(J, ro["J"], rtol=RTOL, atol=0)


def test_context_usable_after_invalid_call(R, oracle_mod):
    p = W.random_slab(6, 5, 4, n_theta=4, n_phi=4, seed=94)
    with R.Solver(p) as s:
        bad = p.chi.copy()
        bad[0, 0, 0] = -1.0
        with pytest.raises(R.RtError):
            R.rt_set_opacity(s.ctx, bad)
        J, _ = s.formal_solution(p.B, want_lstar=False)
    Jo, _ = oracle_mod.formal_solution(p, p.B, lstar=False)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0)
