"""GPU FP32-sweep ("precision") form.

The march runs in FP32 on the deviation I - S_0 from the voxel's own
source, with S held as an FP32 (hi, lo) pair; J, Lambda*, the operator
splitting and the convergence test stay FP64 (Sect. 3.1: small eps needs
double precision for the operator-splitting equations).  Checks: the
formal solution against the FP64 oracle; Lambda* identical to the FP64
path's; converged J against the FP64 path within 1e-6 relative, including
strong scattering (eps = 1e-6), where a march that accumulates I itself in
FP32 would be off by ~1e-3.
"""

import numpy as np
import pytest

from paper_1107_5719_gb300 import workloads as W

pytestmark = pytest.mark.gpu

FS_RTOL = 1e-6       # one formal solution, FP32 march
CONV_RTOL = 1e-6     # converged J, FP32 sweep vs FP64
TOL32 = 5e-8         # outer tolerance the FP32 sweep reaches (its delta floor is ~1e-8)
NG32 = dict(ng_period=4, ng_min_delta=1e-6)   # extrapolate only above the noise


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


@pytest.mark.parametrize("shape,seed", [((17, 9, 6), 1), ((5, 5, 5), 2), ((3, 3, 4), 3),
                                        ((4, 3, 2), 4), ((13, 11, 9), 5)])
def test_fs32_matches_oracle(R, oracle_mod, shape, seed):
    nx, ny, nz = shape
    p = W.random_slab(nx, ny, nz, n_theta=6, n_phi=5, seed=seed, chi_decades=5.0)
    rng = np.random.default_rng(seed)
    S = 0.5 + 2.0 * rng.random(p.B.shape)
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        J, L = s.formal_solution(S)
    Jo, Lo = oracle_mod.formal_solution(p, S)
    assert np.allclose(J, Jo, rtol=FS_RTOL, atol=0)
    # Lambda* is built in FP64 in both forms
    scale = np.abs(Lo).reshape(27, -1).max(axis=0)
    assert np.all(np.abs(L - Lo).reshape(27, -1).max(axis=0) <= 1e-12 * scale)


@pytest.mark.parametrize("top,bottom", [(W.BC_PLANCK, W.BC_ZERO), (W.BC_ZERO, W.BC_DIFFUSION)])
def test_fs32_both_boundary_modes_and_spacings(R, oracle_mod, top, bottom):
    p = W.random_slab(11, 7, 8, n_theta=4, n_phi=6, seed=9, top_bc=top,
                      bottom_bc=bottom, dx=0.6, dy=1.4, dz=0.8)
    S = p.B * 0.7
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        J, _ = s.formal_solution(S, want_lstar=False)
    Jo, _ = oracle_mod.formal_solution(p, S, lstar=False)
    assert np.allclose(J, Jo, rtol=FS_RTOL, atol=0)


def test_fs32_constant_source_is_exact_at_depth(R):
    """S = B = const with a Planck inner boundary: I - S_0 = T_M (B - S_0) = 0
    on every upward ray, so the FP32 march returns J = S exactly where the
    downward rays are fully absorbed."""
    p = W.slab_small(n_theta=8, n_phi=4)
    S = np.ones_like(p.B)
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        J, _ = s.formal_solution(S, want_lstar=False)
    assert np.allclose(J[-3:], 1.0, rtol=1e-15, atol=0)


def test_fs32_deterministic(R):
    """J does not depend on the launch shape: direction groups, threads per
    block and block order (odd ny: the last row of voxel pairs is half
    empty)."""
    p = W.random_slab(19, 9, 7, n_theta=8, n_phi=6, seed=12)
    out = []
    for groups, threads, order in ((0, 0, 0), (1, 64, 2), (4, 128, 1), (8, 256, 2), (2, 256, 0),
                                   (0, 128, 2)):
        with R.Solver(p, precision=R.RT_FP32_SWEEP, groups=groups) as s:
            R.rt_set_block_threads(s.ctx, threads)
            R.rt_set_block_order(s.ctx, order)
            out.append(s.formal_solution(want_lstar=False)[0])
    for J in out[1:]:
        assert np.array_equal(J, out[0])
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        with pytest.raises(R.RtError):
            R.rt_set_block_threads(s.ctx, 96)
        with pytest.raises(R.RtError):
            R.rt_set_block_order(s.ctx, 3)


@pytest.mark.parametrize("eps", [1e-2, 1e-4, 1e-6])
def test_fs32_fixed_point_column_strong_scattering(R, eps):
    """Horizontally uniform 3x3x129 column with the strong-scattering chi law
    (tau 1e-4 .. 1e4): the FP32-sweep iteration, run well past convergence,
    sits within 1e-6 of the FP64 fixed point (measured ~3e-8 on a 9x9x129
    slab at eps = 1e-6)."""
    p = W.slab_precision(n=3, nzz=129, eps=eps, n_theta=16, n_phi=4)
    # the reference marches (its rounding floor at eps = 1e-6 is below 1e-11)
    with R.Solver(p, precision=R.RT_FP64, ng_period=4, record=0) as s:
        r64 = s.solve(tol=1e-11, max_iter=4000)
    assert r64["converged"]
    with R.Solver(p, precision=R.RT_FP32_SWEEP, **NG32) as s:
        R.rt_set_df_finish(s.ctx, 0.0)      # the FP32 sweep alone, at its floor
        r32 = s.solve(tol=0.0, max_iter=max(600, 3 * r64["iters"]))
    rel = np.abs(r32["J"] - r64["J"]) / r64["J"]
    assert rel.max() < CONV_RTOL, rel.max()


def test_fs32_converges_at_its_tolerance(R):
    """The FP32-sweep outer iteration alone (no double-float finish)
    reaches delta < 5e-8 (its rounding floor is ~1e-8) and then agrees with
    the FP64 solution to 1e-6."""
    p = W.slab_small()
    with R.Solver(p, precision=R.RT_FP64) as s:
        r64 = s.solve(tol=1e-10, max_iter=500)
    with R.Solver(p, precision=R.RT_FP32_SWEEP, **NG32) as s:
        R.rt_set_df_finish(s.ctx, 0.0)
        r32 = s.solve(tol=TOL32, max_iter=500)
    assert r32["converged"]
    rel = np.abs(r32["J"] - r64["J"]) / r64["J"]
    assert rel.max() < CONV_RTOL, rel.max()


def test_fs32_slab65_sampled(R, oracle_mod):
    """65^3 slab, 32x32 directions: the FP32-sweep J at sampled voxels
    against the oracle."""
    p = W.slab_65()
    S = p.eps * p.B + (1 - p.eps) * p.B
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        J, _ = s.formal_solution(want_lstar=False)
    rng = np.random.default_rng(6)
    vox = rng.integers(0, p.nvox, 96)
    Jo = oracle_mod.mean_intensity_at(p, S, vox)
    assert np.allclose(J.ravel()[vox], Jo, rtol=FS_RTOL, atol=0)



def test_branch_counts_split_steps_by_segment_optical_depth(R):
    """The diagnostic branch count of the FP32 march: with a uniform opacity
    every segment of direction mu has optical depth chi dz / |mu|, so the
    series branch (x < 2) is taken on every step of the directions with
    chi dz < 2 |mu| and on no step of the others; the step count of each
    direction does not depend on the others (no cutoff)."""
    nx, ny, nz = 9, 8, 7
    base = W.random_slab(nx, ny, nz, seed=41)
    chi = np.full_like(base.chi, 0.5)
    S = base.B * 1.1
    thin = ([0.9, -0.5, 0.35, -0.9], [0.3, 1.7, 2.9, 4.4])   # x = 0.56, 1.0, 1.43, 0.56
    thick = ([0.1, -0.2, 0.15], [0.8, 2.2, 5.1])             # x = 5.0, 2.5, 3.3

    def counts(mu, phi):
        mu, phi = np.array(mu), np.array(phi)
        p = W.Problem(nx, ny, nz, chi, base.eps, base.B, mu, phi, np.full(len(mu), 1 / len(mu)))
        with R.Solver(p, precision=R.RT_FP32_SWEEP, cutoff=0.0, record=0) as s:
            n, ser = R.rt_fs32_branch_counts(s.ctx, S)
            s.formal_solution(S, want_lstar=False)
            assert n == R.rt_last_step_count(s.ctx)
        return n, ser

    n_thin, s_thin = counts(*thin)
    n_thick, s_thick = counts(*thick)
    assert n_thin > 0 and s_thin == n_thin
    assert n_thick > 0 and s_thick == 0
    n_mix, s_mix = counts(thin[0] + thick[0], thin[1] + thick[1])
    assert (n_mix, s_mix) == (n_thin + n_thick, n_thin)


def test_branch_counts_reject_other_precisions(R):
    p = W.random_slab(5, 4, 3, seed=2)
    with R.Solver(p) as s:
        with pytest.raises(R.RtError):
            R.rt_fs32_branch_counts(s.ctx)
