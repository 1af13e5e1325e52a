"""GPU recorded formal solution (FP64 and FP32 sweep) against the oracle.

The first formal solution after the opacities, directions or boundary
change records the march as a linear map of S; later ones replay it for
the new S.  Both must match the oracle to 1e-12 relative in J (FP64 path),
for sources that differ between the recording and the replay, on the same
edge cases as the march itself (ragged tiles, nz = 2, 3x3 planes, both
boundary modes and the LTE-diffusion inner boundary, vertical and grazing
rays), and a converged solve that replays must land on the march's fixed
point.
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


CASES = [
    dict(nx=17, ny=9, nz=6, seed=1),                      # 153-voxel planes: ragged last warp
    dict(nx=3, ny=3, nz=4, seed=3),                        # smallest periodic plane
    dict(nx=4, ny=3, nz=2, seed=4),                        # nz = 2
    dict(nx=13, ny=11, nz=7, seed=5, dx=0.7, dy=1.3, dz=0.9),
    dict(nx=12, ny=7, nz=9, seed=6, top_bc=W.BC_PLANCK, bottom_bc=W.BC_ZERO),
    dict(nx=6, ny=6, nz=8, seed=7, top_bc=W.BC_ZERO, bottom_bc=W.BC_ZERO, chi_decades=6.0),
    dict(nx=10, ny=7, nz=6, seed=8, bottom_bc=W.BC_DIFFUSION),
    dict(nx=5, ny=4, nz=2, seed=9, top_bc=W.BC_PLANCK, bottom_bc=W.BC_DIFFUSION, dz=0.6),
]


def _slab(case):
    kw = dict(case)
    return W.random_slab(kw.pop("nx"), kw.pop("ny"), kw.pop("nz"), n_theta=6, n_phi=5,
                         seed=kw.pop("seed"), **kw)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "{nx}x{ny}x{nz}".format(**c))
def test_record_then_replay_match_oracle(R, oracle_mod, case):
    p = _slab(case)
    rng = np.random.default_rng(11)
    S1 = 0.5 + 2.0 * rng.random(p.B.shape)
    S2 = 0.1 + 5.0 * rng.random(p.B.shape)          # another source: the replay
    with R.Solver(p) as s:
        assert R.rt_fs_record_info(s.ctx) == (0, False)
        J1, _ = s.formal_solution(S1, want_lstar=False)
        nbytes, valid = R.rt_fs_record_info(s.ctx)
        assert nbytes > 0 and valid
        J2, L2 = s.formal_solution(S2)
        J1r, _ = s.formal_solution(S1, want_lstar=False)
    Jo1, _ = oracle_mod.formal_solution(p, S1)
    Jo2, Lo2 = oracle_mod.formal_solution(p, S2)
    assert np.allclose(J1, Jo1, rtol=RTOL, atol=0)
    assert np.allclose(J2, Jo2, rtol=RTOL, atol=0)
    assert np.allclose(J1r, Jo1, rtol=RTOL, atol=0)
    assert np.array_equal(J1r, J1)      # J always comes from the recorded map


def test_special_directions_replay(R, oracle_mod):
    """Vertical, grazing and exact-lattice 45-degree rays through the replay."""
    nx, ny, nz = 7, 5, 6
    mu = np.array([1.0, -1.0, 1e-3, -1e-3, 1 / math.sqrt(2), -1 / math.sqrt(2)])
    phi = np.array([0.3, 1.1, 0.7, 4.0, 0.0, math.pi])
    w = np.full(6, 1 / 6)
    base = W.random_slab(nx, ny, nz, seed=31)
    p = W.Problem(nx, ny, nz, base.chi, base.eps, base.B, mu, phi, w)
    with R.Solver(p) as s:
        s.formal_solution(base.B * 1.3, want_lstar=False)
        J, _ = s.formal_solution(base.B * 0.4 + 0.2, want_lstar=False)
    Jo, _ = oracle_mod.formal_solution(p, base.B * 0.4 + 0.2)
    assert np.allclose(J, Jo, rtol=RTOL, atol=0)


def test_record_off_is_the_march(R):
    """max_bytes 0 (off) and a budget too small to record give the march
    itself, bit for bit, and no recording; the recorded map agrees with the
    march to rounding."""
    p = _slab(CASES[0])
    S = p.B * 0.9 + 0.1
    out = []
    for mode in (0, 1, -1):
        with R.Solver(p) as s:
            R.rt_set_fs_record(s.ctx, mode)
            J, _ = s.formal_solution(S, want_lstar=False)      # the march (records if on)
            out.append(J)
            nbytes, valid = R.rt_fs_record_info(s.ctx)
            assert (nbytes > 0 and valid) == (mode == -1)
    assert np.array_equal(out[0], out[1])
    assert np.allclose(out[2], out[0], rtol=1e-14, atol=0)
    with R.Solver(p) as s:
        with pytest.raises(R.RtError):
            R.rt_set_fs_record(s.ctx, -2)


def test_new_opacity_records_again(R, oracle_mod):
    """A new opacity (or boundary, or cutoff) invalidates the recording: the
    next formal solution marches the new problem and records it."""
    p = _slab(CASES[3])
    q = _slab(dict(CASES[3], seed=55))
    S = p.B * 1.1
    with R.Solver(p) as s:
        s.formal_solution(S, want_lstar=False)
        s.formal_solution(S, want_lstar=False)
        R.rt_set_opacity(s.ctx, q.chi)
        assert R.rt_fs_record_info(s.ctx)[1] is False
        J, _ = s.formal_solution(S, want_lstar=False)
        assert R.rt_fs_record_info(s.ctx)[1] is True
        J2, _ = s.formal_solution(S * 0.5, want_lstar=False)
        R.rt_set_boundary(s.ctx, W.BC_PLANCK, W.BC_PLANCK)
        assert R.rt_fs_record_info(s.ctx)[1] is False
        J3, _ = s.formal_solution(S, want_lstar=False)
        R.rt_set_cutoff(s.ctx, 0.0)
        assert R.rt_fs_record_info(s.ctx)[1] is False
    pq = W.Problem(q.nx, q.ny, q.nz, q.chi, p.eps, p.B, p.mu, p.phi, p.w, dx=q.dx, dy=q.dy,
                   dz=q.dz, top_bc=p.top_bc, bottom_bc=p.bottom_bc)
    assert np.allclose(J, oracle_mod.formal_solution(pq, S)[0], rtol=RTOL, atol=0)
    assert np.allclose(J2, oracle_mod.formal_solution(pq, S * 0.5)[0], rtol=RTOL, atol=0)
    pb = W.Problem(q.nx, q.ny, q.nz, q.chi, p.eps, p.B, p.mu, p.phi, p.w, dx=q.dx, dy=q.dy,
                   dz=q.dz, top_bc=W.BC_PLANCK, bottom_bc=W.BC_PLANCK)
    assert np.allclose(J3, oracle_mod.formal_solution(pb, S)[0], rtol=RTOL, atol=0)


def test_converged_solve_replaying_matches_the_march(R):
    """A converged solve that records once and replays afterwards reaches
    the fixed point of the solve that marches every time."""
    p = W.slab_small(n_theta=8, n_phi=8)
    res = []
    for mode in (0, -1):
        with R.Solver(p, ng_period=4) as s:
            R.rt_set_fs_record(s.ctx, mode)
            res.append(s.solve(tol=1e-12, max_iter=500))
    assert res[0]["converged"] and res[1]["converged"]
    assert np.allclose(res[1]["J"], res[0]["J"], rtol=1e-11, atol=0)
    assert abs(res[1]["iters"] - res[0]["iters"]) <= 1


FS32_RTOL = 1e-6        # one FP32-sweep formal solution against the oracle


@pytest.mark.parametrize("case", CASES, ids=lambda c: "fp32-{nx}x{ny}x{nz}".format(**c))
def test_fp32_record_then_replay_match_oracle(R, oracle_mod, case):
    """The FP32 sweep records its march (difference form) and replays it for
    other sources: both within the FP32 parity of the oracle, and the replay
    of the recording source equal to the recording formal solution."""
    p = _slab(case)
    rng = np.random.default_rng(12)
    S1 = 0.5 + 2.0 * rng.random(p.B.shape)
    S2 = 0.1 + 5.0 * rng.random(p.B.shape)
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        J1, _ = s.formal_solution(S1, want_lstar=False)
        nbytes, valid = R.rt_fs_record_info(s.ctx)
        assert nbytes > 0 and valid
        J2, _ = s.formal_solution(S2, want_lstar=False)
        J1r, _ = s.formal_solution(S1, want_lstar=False)
    assert np.array_equal(J1r, J1)
    assert np.allclose(J1, oracle_mod.formal_solution(p, S1)[0], rtol=FS32_RTOL, atol=0)
    assert np.allclose(J2, oracle_mod.formal_solution(p, S2)[0], rtol=FS32_RTOL, atol=0)


def test_fp32_replay_agrees_with_the_march(R):
    p = W.random_slab(21, 13, 9, n_theta=6, n_phi=5, seed=17, chi_decades=5.0)
    S = 0.3 + np.random.default_rng(3).random(p.B.shape)
    out = []
    for mode in (0, -1):
        with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
            R.rt_set_fs_record(s.ctx, mode)
            s.formal_solution(p.B, want_lstar=False)              # records (mode -1)
            out.append(s.formal_solution(S, want_lstar=False)[0])
    assert np.allclose(out[1], out[0], rtol=2e-7, atol=0)


def test_fp32_solve_through_the_replay_meets_fp64(R):
    """The FP32 form as created (finishing stage from delta < 1e-6; its
    source-change marches replay the recording with zero boundary
    intensities) converges to the FP64 fixed point within 1e-6, as the
    marching solve does."""
    p = W.slab_precision(n=5, nzz=33, eps=1e-4, n_theta=8, n_phi=4)
    with R.Solver(p, precision=R.RT_FP64, ng_period=4, record=0) as s:
        r64 = s.solve(tol=1e-11, max_iter=3000)
    res = []
    for mode in (0, -1):
        with R.Solver(p, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
            R.rt_set_fs_record(s.ctx, mode)
            res.append(s.solve(tol=1e-9, max_iter=3000))
            assert R.rt_fs_record_info(s.ctx)[1] == (mode == -1)
    for r in res:
        assert r["converged"]
        assert np.max(np.abs(r["J"] - r64["J"]) / r64["J"]) < 1e-6
    assert np.max(np.abs(res[1]["J"] - res[0]["J"]) / res[0]["J"]) < 1e-7


PARA_CASES = [c for c in CASES if c.get("chi_decades", 3.0) <= 3.0]


@pytest.mark.parametrize("case", PARA_CASES, ids=lambda c: "para-{nx}x{ny}x{nz}".format(**c))
def test_parabolic_record_then_replay_match_oracle(R, oracle_mod, case):
    """The parabolic source records its march too (the coefficient of S at
    the downstream point p_-1 beside those of the upstream points): the
    recording and the replay of another source against the oracle."""
    p = _slab(case)
    p.src_order = 1
    rng = np.random.default_rng(13)
    S1 = 0.5 + 2.0 * rng.random(p.B.shape)
    S2 = 0.1 + 5.0 * rng.random(p.B.shape)
    with R.Solver(p) as s:
        J1, _ = s.formal_solution(S1, want_lstar=False)
        assert R.rt_fs_record_info(s.ctx)[1]
        J2, _ = s.formal_solution(S2, want_lstar=False)
    with R.Solver(p, record=0) as s:
        J2m, _ = s.formal_solution(S2, want_lstar=False)
    assert np.allclose(J1, oracle_mod.formal_solution(p, S1)[0], rtol=RTOL, atol=0)
    assert np.allclose(J2, oracle_mod.formal_solution(p, S2)[0], rtol=RTOL, atol=0)
    assert np.allclose(J2, J2m, rtol=1e-13, atol=0)


@pytest.mark.parametrize("case", CASES, ids=lambda c: "df-{nx}x{ny}x{nz}".format(**c))
def test_double_float_record_then_replay_match_oracle(R, oracle_mod, case):
    """The double-float form records its march (double-float coefficients
    of S(p_m) - S_0) and replays it: both within the FP64 bar of the oracle,
    and the replay of the recording source equal to the recording solution."""
    p = _slab(case)
    rng = np.random.default_rng(14)
    S1 = 0.5 + 2.0 * rng.random(p.B.shape)
    S2 = 0.1 + 5.0 * rng.random(p.B.shape)
    with R.Solver(p, precision=R.RT_DF64) as s:
        J1, _ = s.formal_solution(S1, want_lstar=False)
        assert R.rt_fs_record_info(s.ctx)[1]
        J2, _ = s.formal_solution(S2, want_lstar=False)
        J1r, _ = s.formal_solution(S1, want_lstar=False)
    assert np.array_equal(J1r, J1)
    assert np.allclose(J1, oracle_mod.formal_solution(p, S1)[0], rtol=RTOL, atol=0)
    assert np.allclose(J2, oracle_mod.formal_solution(p, S2)[0], rtol=RTOL, atol=0)
