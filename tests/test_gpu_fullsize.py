"""Parity at the full size of the strong-scattering slab: 129^3 voxels, 64x64
directions, eps = 1e-6, in the launch configuration of the library's own
solves.  The oracle computes J at sampled voxels (every plane plus random
ones), one characteristic at a time."""

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


@pytest.fixture(scope="module")
def case(oracle_mod):
    p = W.slab_precision()                     # 129^3, 64x64 directions
    rng = np.random.default_rng(17)
    S = 0.5 + rng.random(p.B.shape)            # a source with structure in every direction
    ks = np.concatenate([np.arange(p.nz), rng.integers(0, p.nz, 31)])
    vox = ks * p.nx * p.ny + rng.integers(0, p.nx * p.ny, ks.shape[0])
    Jo = oracle_mod.mean_intensity_at(p, S, vox)
    return p, S, vox, Jo


@pytest.mark.parametrize("prec,rtol", [("fp64", 1e-12), ("df64", 1e-12), ("fp32", 1e-6)])
def test_slab129_formal_solution_sampled(R, case, prec, rtol):
    p, S, vox, Jo = case
    precision = {"fp64": R.RT_FP64, "df64": R.RT_DF64, "fp32": R.RT_FP32_SWEEP}[prec]
    with R.Solver(p, precision=precision) as s:
        J, _ = s.formal_solution(S, want_lstar=False)
    Js = J.ravel()[vox]
    assert np.allclose(Js, Jo, rtol=rtol, atol=0), np.max(np.abs(Js - Jo) / Jo)


def test_uneven_batch_largest_grid_sampled(R, oracle_mod):
    """The largest grid of the uneven batch, 257 x 257 x 129 with 64x64
    directions (one wavelength of it), FP32 sweep and double-float march,
    J at sampled voxels against the oracle."""
    q = W.batch_uneven(sizes=((257, 257, 129, 1),))[0]
    rng = np.random.default_rng(23)
    S = 0.5 + rng.random(q.chi.shape)
    ks = np.concatenate([np.arange(0, q.nz, 4), rng.integers(0, q.nz, 15)])
    vox = ks * q.nx * q.ny + rng.integers(0, q.nx * q.ny, ks.shape[0])
    Jo = oracle_mod.mean_intensity_at(q, S, vox)
    for precision, rtol in ((R.RT_DF64, 1e-12), (R.RT_FP32_SWEEP, 1e-6)):
        with R.Solver(q, precision=precision) as s:
            J, _ = s.formal_solution(S, want_lstar=False)
        Js = J.ravel()[vox]
        assert np.allclose(Js, Jo, rtol=rtol, atol=0), (precision, np.max(np.abs(Js - Jo) / Jo))
