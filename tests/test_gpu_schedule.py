"""Plane dispatch order of the FP64 march launches: it is the permutation the
work estimate defines (plane means of chi marched to an optical depth of 40
at |mu| = 1, 1/2, 1/5), it follows the opacity, and it changes no result."""

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


def _work(chi, dz):
    """The estimate, restated on the host."""
    nz = chi.shape[0]
    mean = chi.reshape(nz, -1).mean(axis=1)
    work = np.zeros(nz)
    for k0 in range(nz):
        for amu in (1.0, 0.5, 0.2):
            hs = dz / (2.0 * amu)
            for s in (-1, 1):
                tau, n, k = 0.0, 1, k0
                while 0 <= k - s < nz and tau <= 40.0:
                    tau += hs * (mean[k] + mean[k - s])
                    k -= s
                    n += 1
                work[k0] += n
    return work


def _order(R, p):
    ctx = R.rt_create(0, R.RT_FP64)
    try:
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_opacity(ctx, p.chi)
        return R.rt_get_plane_order(ctx, p.nz)
    finally:
        R.rt_destroy(ctx)


def _check_order(order, work):
    nz = len(work)
    assert sorted(order.tolist()) == list(range(nz))
    # non-increasing estimated work; the host and device plane means differ
    # in summation order, which can move a step count by one at tau = 40
    w = work[order]
    assert np.all(w[1:] <= w[:-1] + 1)


def test_order_of_a_slab_puts_the_transparent_planes_first(R):
    p = W.slab_65(n=33, n_theta=4, n_phi=4)
    order = _order(R, p)
    work = _work(p.chi, p.dz)
    _check_order(order, work)
    # chi grows with depth: the opaque bottom planes (characteristics end
    # after a step or two) are dispatched last
    assert set(order[-8:].tolist()) <= set(range(p.nz - 12, p.nz))


def test_order_follows_the_opacity(R):
    p = W.slab_65(n=33, n_theta=4, n_phi=4)
    p.chi = np.ascontiguousarray(p.chi[::-1])
    order = _order(R, p)
    _check_order(order, _work(p.chi, p.dz))
    assert set(order[-8:].tolist()) <= set(range(12))


@pytest.mark.parametrize("flip", [False, True])
def test_order_changes_no_result(R, flip):
    """J of a context (estimated order, autotuned groups) is bit-identical
    to J of the allocation-free call (planes in index order)."""
    import torch
    p = W.slab_65(n=21, n_theta=4, n_phi=6)
    if flip:
        p.chi = np.ascontiguousarray(p.chi[::-1])
    if flip:
        assert not np.array_equal(_order(R, p), np.arange(p.nz))
    dev = torch.device("cuda:0")
    S = p.B * (1.0 + 0.1 * np.random.default_rng(5).random(p.B.shape))
    with R.Solver(p, record=0) as s:      # the allocation-free entry marches
        Jc, _ = s.formal_solution(S)
    J = torch.empty(p.B.shape, dtype=torch.float64, device=dev)
    rc = R.rt_formal_solution_noalloc(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.top_bc, p.bottom_bc,
                                      p.mu, p.phi, p.w, torch.from_numpy(p.chi).to(dev),
                                      torch.from_numpy(S).to(dev), torch.from_numpy(p.B).to(dev), J)
    torch.cuda.synchronize()
    assert rc == R.RT_OK
    assert np.array_equal(J.cpu().numpy(), Jc)
