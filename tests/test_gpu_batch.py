"""Batched wavelengths: many problems, one fused formal-solution launch per
outer iteration (FP32 sweep), per-problem convergence.

Each problem's iterates must be exactly those of solving it alone with the
same precision (same arithmetic per voxel, fixed summation order), so J is
compared bit for bit; problems of different grid sizes (an uneven batch)
share the launch.  The FP64 batch is checked against the oracle.
"""

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


def _uneven(n_theta=6, n_phi=4):
    probs = []
    for i, (nx, ny, nz) in enumerate([(9, 7, 6), (17, 9, 11), (5, 5, 5), (13, 11, 9), (3, 3, 4)]):
        p = W.random_slab(nx, ny, nz, n_theta=n_theta, n_phi=n_phi, seed=200 + i,
                          eps_range=(10 ** (-1 - i), 1.0))
        probs.append(p)
    return probs


# FP32 sweep: the iterate's delta floor is ~1e-8 with many directions and
# higher with the few directions used here; equality with the individual
# solves holds at any tolerance.
TOL = {1: 1e-6, 0: 1e-9}


@pytest.mark.parametrize("record", [-1, 0], ids=["recorded", "marching"])
@pytest.mark.parametrize("precision", [1, 0])
def test_batch_equals_individual_solves(R, precision, record):
    """Bit-identical to single solves, with the recorded march (record once,
    replay in the fused launch) and without."""
    probs = _uneven()
    b = R.rt_batch_create(probs, precision=precision)
    try:
        R.rt_batch_set_ng(b, 4, 1e-6)
        R.rt_batch_set_fs_record(b, record)
        r = R.rt_batch_solve(b, len(probs), tol=TOL[precision], max_iter=500)
        assert r["converged"] and r["n_converged"] == len(probs)
        for i, p in enumerate(probs):
            J = R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx))
            with R.Solver(p, precision=precision, ng_period=4, ng_min_delta=1e-6,
                          record=record) as s:
                ri = s.solve(tol=TOL[precision], max_iter=500)
            assert ri["iters"] == r["iters"][i]
            assert np.array_equal(J, ri["J"]), i
        st = R.rt_batch_get_stats(b)
        assert st["fs_launches"] == (max(r["iters"]) if precision == 1 else int(r["iters"].sum()))
    finally:
        R.rt_batch_destroy(b)


def test_batch_recordings_in_waves(R):
    """A budget that holds two recordings at a time: the problems run in
    waves (each starts once memory frees), with the iterates of single
    solves, bit for bit; the recordings' memory returns at the end."""
    probs = _uneven()[:5]
    sizes = []
    for p in probs:
        with R.Solver(p, precision=1) as s:
            s.formal_solution(p.B, want_lstar=False)
            sizes.append(R.rt_fs_record_info(s.ctx)[0])
    b = R.rt_batch_create(probs, precision=1)
    try:
        R.rt_batch_set_ng(b, 4, 1e-6)
        R.rt_batch_set_fs_record(b, sum(sorted(sizes)[-2:]))
        r = R.rt_batch_solve(b, len(probs), tol=TOL[1], max_iter=500)
        assert r["converged"]
        st = R.rt_batch_get_stats(b)
        assert st["iterations"] > max(r["iters"])        # more than one wave
        for i, p in enumerate(probs):
            with R.Solver(p, precision=1, ng_period=4, ng_min_delta=1e-6) as s:
                ri = s.solve(tol=TOL[1], max_iter=500)
            assert ri["iters"] == r["iters"][i]
            assert np.array_equal(R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx)), ri["J"]), i
    finally:
        R.rt_batch_destroy(b)
    b = R.rt_batch_create(probs[:1], precision=1)
    try:
        with pytest.raises(R.RtError):
            R.rt_batch_set_fs_record(b, -5)
    finally:
        R.rt_batch_destroy(b)


def test_batch_fp64_matches_oracle(R, oracle_mod):
    probs = _uneven(n_theta=4, n_phi=4)[:3]
    b = R.rt_batch_create(probs, precision=0)
    try:
        r = R.rt_batch_solve(b, len(probs), tol=1e-9, max_iter=500, tol_inner=0.0, max_sweeps=10)
        for i, p in enumerate(probs):
            ro = oracle_mod.solve(p, tol=1e-9, max_iter=500, tol_inner=0.0, max_sweeps=10)
            assert ro["iters"] == r["iters"][i]
            J = R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx))
            assert np.allclose(J, ro["J"], rtol=1e-12, atol=0)
    finally:
        R.rt_batch_destroy(b)


def test_batch_reset_and_restart(R):
    probs = _uneven()[:3]
    b = R.rt_batch_create(probs, precision=1)
    try:
        r1 = R.rt_batch_solve(b, 3, tol=TOL[1], max_iter=500)
        J1 = [R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx)) for i, p in enumerate(probs)]
        R.rt_batch_reset(b, rebuild_lstar=True)
        r2 = R.rt_batch_solve(b, 3, tol=TOL[1], max_iter=500)
        J2 = [R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx)) for i, p in enumerate(probs)]
        assert np.array_equal(r1["iters"], r2["iters"])
        for a, c in zip(J1, J2):
            assert np.array_equal(a, c)
    finally:
        R.rt_batch_destroy(b)


def test_batch_wavelengths_of_one_slab(R):
    """A small wavelength batch built like the 512-point one (65^3 slab
    scaled per wavelength), reduced to 8 points on a 17^3 slab: the batch
    converges every point and matches per-point FP32 solves."""
    probs = W.batch_65(n_lambda=8, n=17, n_theta=8, n_phi=4)
    b = R.rt_batch_create(probs, precision=1)
    try:
        R.rt_batch_set_ng(b, 4, 1e-6)
        r = R.rt_batch_solve(b, len(probs), tol=TOL[1], max_iter=2000)
        assert r["converged"]
        for i in (0, 5):
            with R.Solver(probs[i], precision=1, ng_period=4, ng_min_delta=1e-6) as s:
                ri = s.solve(tol=TOL[1], max_iter=2000)
            J = R.rt_batch_get_J(b, i, ri["J"].shape)
            assert np.array_equal(J, ri["J"])
    finally:
        R.rt_batch_destroy(b)


@pytest.mark.parametrize("method", [0, 1])
def test_batch_graph_equals_host_loop(R, method):
    """The operator-splitting step of all active problems as one CUDA graph
    (per-problem branches with device-side sweep loops) gives the iterates
    of the host-driven sweep chunks bit for bit, Jacobi and red-black
    Gauss-Seidel, with one host wait per iteration (Ng on the device too)
    instead of one per chunk of sweeps."""
    probs = _uneven()
    out = {}
    for graphs in (True, False):
        b = R.rt_batch_create(probs, precision=1)
        try:
            R.rt_batch_set_graphs(b, graphs)
            R.rt_batch_set_os_method(b, method)
            R.rt_batch_set_ng(b, 4, 1e-6)
            r = R.rt_batch_solve(b, len(probs), tol=TOL[1], max_iter=500)
            assert r["converged"]
            Js = [R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx)) for i, p in enumerate(probs)]
            out[graphs] = (r, Js, R.rt_batch_get_stats(b))
        finally:
            R.rt_batch_destroy(b)
    (rg, Jg, sg), (rh, Jh, sh) = out[True], out[False]
    assert np.array_equal(rg["iters"], rh["iters"])
    for a, c in zip(Jg, Jh):
        assert np.array_equal(a, c)
    assert sg["iterations"] == sh["iterations"] == max(rg["iters"])
    assert sg["host_syncs"] == sg["iterations"]        # one wait per outer iteration
    assert sh["host_syncs"] > sg["host_syncs"]


def test_batch_launch_shape_does_not_change_results(R):
    """Threads per block, direction groups and block order of the fused FP32
    launch are tuning knobs only: bit-identical iterates."""
    probs = _uneven()[:3]
    out = []
    for groups, threads, order in ((0, 0, 0), (2, 64, 2), (8, 256, 1), (1, 128, 2)):
        b = R.rt_batch_create(probs, precision=1)
        try:
            R.rt_batch_set_direction_groups(b, groups)
            R.rt_batch_set_block_threads(b, threads)
            R.rt_batch_set_block_order(b, order)
            r = R.rt_batch_solve(b, len(probs), tol=TOL[1], max_iter=500)
            out.append((r["iters"], [R.rt_batch_get_J(b, i, (p.nz, p.ny, p.nx))
                                     for i, p in enumerate(probs)]))
        finally:
            R.rt_batch_destroy(b)
    for it, Js in out[1:]:
        assert np.array_equal(it, out[0][0])
        for a, c in zip(Js, out[0][1]):
            assert np.array_equal(a, c)
