"""Switching a context between the FP32 sweep and the double-float march
(rt_set_precision): the strong-scattering column (eps = 1e-6) solved with
the FP32 sweep to its tolerance stands ~4e-6 from the FP64 fixed point
(the outer iteration contracts slowly); a few double-float iterations with
Ng on bring it within 1e-6."""

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


def test_fp32_then_double_float_reaches_1e6(R):
    p = W.slab_precision(n=9, nzz=129, n_theta=32, n_phi=8)
    # the reference marches (its rounding floor at eps = 1e-6 is below 1e-11)
    with R.Solver(p, precision=R.RT_FP64, ng_period=4, record=0) as s:
        r64 = s.solve(tol=1e-11, max_iter=5000)
    assert r64["converged"]
    with R.Solver(p, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
        R.rt_set_df_finish(s.ctx, 0.0)          # the FP32 sweep alone, switched by hand
        r32 = s.solve(tol=5e-8, max_iter=5000)
        assert r32["converged"]
        err32 = np.max(np.abs(r32["J"] - r64["J"]) / r64["J"])
        R.rt_set_precision(s.ctx, R.RT_DF64)
        R.rt_set_ng(s.ctx, 4, 0.0)
        rdf = s.solve(tol=1e-8, max_iter=200)
        assert rdf["converged"]
        errdf = np.max(np.abs(rdf["J"] - r64["J"]) / r64["J"])
    assert err32 > 1e-6          # the stopping error the finish removes
    assert errdf < 1e-6, (err32, errdf)
    assert rdf["iters"] < 0.05 * r32["iters"]


def test_precision_switch_round_trip(R):
    """After a switch the formal solution is the one of a context created in
    that precision, bit for bit, in both directions."""
    p = W.random_slab(13, 11, 7, n_theta=6, n_phi=5, seed=5, bottom_bc=W.BC_DIFFUSION)
    S = p.B * 1.1
    ref = {}
    for prec in (R.RT_FP32_SWEEP, R.RT_DF64):
        with R.Solver(p, precision=prec) as s:
            ref[prec] = s.formal_solution(S)
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        for prec in (R.RT_DF64, R.RT_FP32_SWEEP, R.RT_DF64):
            R.rt_set_precision(s.ctx, prec)
            J, L = s.formal_solution(S)
            assert np.array_equal(J, ref[prec][0])
            assert np.array_equal(L, ref[prec][1])
        with pytest.raises(R.RtError):
            R.rt_set_precision(s.ctx, R.RT_FP64)
    with R.Solver(p, precision=R.RT_FP64) as s:
        with pytest.raises(R.RtError):
            R.rt_set_precision(s.ctx, R.RT_DF64)


def test_batch_fp32_then_double_float_equals_single(R):
    """The batch's two stages (fused FP32 launches, then per-problem
    double-float launches) give each problem the iterates of solving it
    alone with the same two stages."""
    probs = [W.slab_precision(n=7, nzz=33, eps=e, n_theta=8, n_phi=4, seed=70 + i)
             for i, e in enumerate((1e-6, 1e-4, 1e-2))]
    b = R.rt_batch_create(probs, precision=R.RT_FP32_SWEEP)
    try:
        R.rt_batch_set_ng(b, 4, 1e-6)
        R.rt_batch_set_df_finish(b, 0.0)        # stages switched by hand
        r1 = R.rt_batch_solve(b, len(probs), tol=5e-8, max_iter=3000)
        assert r1["converged"]
        R.rt_batch_set_precision(b, R.RT_DF64)
        R.rt_batch_set_ng(b, 4, 0.0)
        r2 = R.rt_batch_solve(b, len(probs), tol=1e-8, max_iter=500)
        assert r2["converged"]
        Jb = [R.rt_batch_get_J(b, i, (q.nz, q.ny, q.nx)) for i, q in enumerate(probs)]
    finally:
        R.rt_batch_destroy(b)
    for i, q in enumerate(probs):
        with R.Solver(q, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
            R.rt_set_df_finish(s.ctx, 0.0)
            a = s.solve(tol=5e-8, max_iter=3000)
            R.rt_set_precision(s.ctx, R.RT_DF64)
            R.rt_set_ng(s.ctx, 4, 0.0)
            c = s.solve(tol=1e-8, max_iter=500)
        assert a["iters"] == r1["iters"][i] and c["iters"] == r2["iters"][i]
        assert np.array_equal(c["J"], Jb[i])


def test_automatic_double_float_finish(R):
    """rt_set_df_finish (on by default for FP32-sweep contexts): the
    FP32-sweep solve switches itself to double-float once delta < 1e-6 and
    reaches a tolerance below the FP32 noise floor, in fewer iterations than
    the FP32 sweep alone needs for 5e-8; afterwards the context is an
    FP32-sweep context again."""
    p = W.slab_precision(n=9, nzz=129, n_theta=32, n_phi=8)
    # the reference marches (its rounding floor at eps = 1e-6 is below 1e-11)
    with R.Solver(p, precision=R.RT_FP64, ng_period=4, record=0) as s:
        r64 = s.solve(tol=1e-11, max_iter=5000)
    with R.Solver(p, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
        R.rt_set_df_finish(s.ctx, 0.0)
        r32 = s.solve(tol=5e-8, max_iter=5000)
    S = p.B * 1.1
    with R.Solver(p, precision=R.RT_FP32_SWEEP) as s:
        Jref, _ = s.formal_solution(S)
    with R.Solver(p, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
        r = s.solve(tol=1e-8, max_iter=5000)        # the context's default finish
        J, _ = s.formal_solution(S)                 # back in the FP32 sweep
    assert r["converged"]
    err = np.max(np.abs(r["J"] - r64["J"]) / r64["J"])
    assert err < 1e-6, err
    assert r["iters"] < r32["iters"]
    assert np.array_equal(J, Jref)


def test_batch_automatic_finish_equals_single(R):
    probs = [W.slab_precision(n=7, nzz=33, eps=e, n_theta=8, n_phi=4, seed=80 + i)
             for i, e in enumerate((1e-6, 1e-4, 1e-2))]
    b = R.rt_batch_create(probs, precision=R.RT_FP32_SWEEP)
    try:
        R.rt_batch_set_ng(b, 4, 1e-6)
        R.rt_batch_set_df_finish(b, 1e-6)
        rb = R.rt_batch_solve(b, len(probs), tol=1e-8, max_iter=3000)
        assert rb["converged"]
        Jb = [R.rt_batch_get_J(b, i, (q.nz, q.ny, q.nx)) for i, q in enumerate(probs)]
    finally:
        R.rt_batch_destroy(b)
    for i, q in enumerate(probs):
        with R.Solver(q, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
            R.rt_set_df_finish(s.ctx, 1e-6)
            r = s.solve(tol=1e-8, max_iter=3000)
        assert r["iters"] == rb["iters"][i]
        assert np.array_equal(r["J"], Jb[i])


@pytest.mark.parametrize("eps", [1e-2, 1e-4])
def test_finishing_stage_is_fp64_accurate(R, eps):
    """After the switch the FP32-sweep context's formal solutions are
    J_ref + J_FS(S - S_ref), the reference in double-float and the change in
    FP32: accurate enough to iterate to delta < 1e-10, two orders below the
    FP32 sweep's own floor, and to land on the double-float fixed point."""
    p = W.random_slab(13, 11, 17, n_theta=8, n_phi=6, seed=33, eps_range=(eps, eps),
                      chi_decades=4.0)
    with R.Solver(p, precision=R.RT_DF64, ng_period=4) as s:
        rdf = s.solve(tol=1e-11, max_iter=3000)
    assert rdf["converged"]
    with R.Solver(p, precision=R.RT_FP32_SWEEP, ng_period=4, ng_min_delta=1e-6) as s:
        r = s.solve(tol=1e-10, max_iter=3000)
    assert r["converged"]
    err = np.max(np.abs(r["J"] - rdf["J"]) / rdf["J"])
    assert err < 1e-8, err
