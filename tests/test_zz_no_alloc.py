"""The allocation-free formal solution against the context-based one.

rt_formal_solution_noalloc serves callers that may not allocate device
memory while they run: a plug-in whose host application owns every device
allocation, a service whose memory budget is fixed up front, or code that
cannot afford the device-wide synchronisation a cudaMalloc can cause.  It
works in one fixed device array owned by the library instead of a
context's buffers, and that array keeps whatever the previous call left in
it.  So this test makes two calls in a row, on different grids, boundary
modes and sources, and checks each against rt_formal_solution_dev at the
FP64 tolerance of the other GPU tests.  The file name makes pytest collect
it last.
"""

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


def _context_fs(R, p, S):
    import torch
    dev = torch.device("cuda:0")
    ctx = R.rt_create(0, R.RT_FP64)
    try:
        R.rt_set_grid(ctx, p.nx, p.ny, p.nz, p.dx, p.dy, p.dz)
        R.rt_set_boundary(ctx, p.top_bc, p.bottom_bc)
        R.rt_set_quadrature(ctx, p.mu, p.phi, p.w)
        R.rt_set_opacity(ctx, p.chi)
        R.rt_set_epsilon(ctx, p.eps)
        R.rt_set_planck(ctx, p.B)
        J = torch.empty(p.B.shape, dtype=torch.float64, device=dev)
        R.rt_formal_solution_dev(ctx, torch.from_numpy(S).to(dev), J, None)
        torch.cuda.synchronize()
        return J.cpu().numpy()
    finally:
        R.rt_destroy(ctx)


def _noalloc_fs(R, p, S):
    import torch
    dev = torch.device("cuda:0")
    chi = torch.from_numpy(p.chi).to(dev)
    St = torch.from_numpy(S).to(dev)
    B = torch.from_numpy(p.B).to(dev)
    J = torch.full(p.B.shape, float("nan"), dtype=torch.float64, device=dev)
    stream = torch.cuda.current_stream()
    rc = R.rt_formal_solution_noalloc(p.nx, p.ny, p.nz, p.dx, p.dy, p.dz, p.top_bc, p.bottom_bc,
                                      p.mu, p.phi, p.w, chi, St, B, J, stream)
    assert rc == R.RT_OK, rc
    stream.synchronize()
    return J.cpu().numpy()


def test_noalloc_matches_context_path_on_two_calls_in_a_row(R):
    first = W.random_slab(17, 9, 6, n_theta=6, n_phi=5, seed=101, chi_decades=5.0)
    second = W.random_slab(11, 13, 9, n_theta=4, n_phi=7, seed=102, top_bc=W.BC_PLANCK,
                           bottom_bc=W.BC_ZERO, dx=0.8, dy=1.2, dz=0.9)
    rng = np.random.default_rng(7)
    S1 = 1.0 + 3.0 * rng.random(first.B.shape)
    S2 = 0.1 + 0.2 * rng.random(second.B.shape)   # smaller source bound than the first call
    for p, S in ((first, S1), (second, S2)):
        J_ref = _context_fs(R, p, S)
        J = _noalloc_fs(R, p, S)
        assert np.all(np.isfinite(J))
        assert np.allclose(J, J_ref, rtol=RTOL, atol=0)


def test_noalloc_rejects_what_does_not_fit_or_is_invalid(R):
    import torch
    dev = torch.device("cuda:0")
    x = torch.ones(8, dtype=torch.float64, device=dev)
    mu, phi, w = W.quadrature(4, 4)
    # 257 x 257 x 129 voxels need 545 MB of partial sums: more than the scratch
    rc = R.rt_formal_solution_noalloc(257, 257, 129, 1.0, 1.0, 1.0, 0, 1, mu, phi, w, x, x, x, x)
    assert rc == R.RT_ESCRATCH
    rc = R.rt_formal_solution_noalloc(2, 5, 5, 1.0, 1.0, 1.0, 0, 1, mu, phi, w, x, x, x, x)
    assert rc == R.RT_EINVAL
    rc = R.rt_formal_solution_noalloc(5, 5, 5, 1.0, 1.0, 1.0, 0, 1, mu, phi, w * 2.0, x, x, x, x)
    assert rc == R.RT_EINVAL
