"""The recorded formal solution's coefficients, checked on the CPU against
the oracle's own march.

For fixed opacities the intensity of a characteristic is linear in the
source (Sect. 2.2).  The recording kernels store, per (voxel, direction),
the coefficient of S at every point of the ray; these tests rebuild those
coefficients in plain Python from the oracle's segment weights, exactly by
the rules the recording kernels follow, and require that they reproduce
the oracle's intensity for random sources on vertical rays (whose points
are voxel centres, so no interpolation enters):

  linear:    c_0 = w_cur,0,  c_m = T_{m-1} w_up,m-1 + T_m w_cur,m,
             c_M = T_{M-1} w_up,M-1,  I = sum_m c_m S_m + T_M I_bc;
  parabolic: segment m adds T_m P_up, T_m P_cur, T_m P_down to the
             coefficients of p_{m+1}, p_m, p_{m-1} (the first segment
             without a downstream point takes the linear weights);

and that the difference form the FP32 and double-float recordings replay,
I - S_0 = sum_{m>=1} c_m (S_m - S_0) + T_M (I_bc - S_0), holds because the
coefficients and T_M sum to one.
"""

import math

import numpy as np
import pytest

from paper_1107_5719_gb300 import workloads as W


def _column_problem(nz, top_bc, bottom_bc, seed, src_order=0):
    rng = np.random.default_rng(seed)
    nx = ny = 3
    chi = 10.0 ** rng.uniform(-2, 1, (nz, ny, nx))
    eps = np.full((nz, ny, nx), 0.1)
    B = 1.0 + rng.random((nz, ny, nx))
    p = W.Problem(nx, ny, nz, chi, eps, B, np.array([1.0]), np.array([0.0]), np.array([1.0]),
                  dz=0.7, top_bc=top_bc, bottom_bc=bottom_bc)
    p.src_order = src_order
    return p


def _ray(p, sgn, i, j, k0):
    """Points p_0 = (i, j, k0), p_m on plane k0 - m sgn up to the boundary
    plane; segment optical depths by the trapezoid rule."""
    M = k0 if sgn > 0 else p.nz - 1 - k0
    ks = [k0 - m * sgn for m in range(M + 1)]
    hs = p.dz / 2.0
    x = [hs * (p.chi[ks[m], j, i] + p.chi[ks[m + 1], j, i]) for m in range(M)]
    return ks, x


def _linear_coefficients(oracle_mod, x):
    M = len(x)
    c = np.zeros(M + 1)
    T = 1.0
    for m in range(M):
        wc, wu = oracle_mod.weights(x[m])
        c[m] += T * wc
        c[m + 1] += T * wu
        T *= math.exp(-x[m])
    return c, T


@pytest.mark.parametrize("sgn", [1, -1])
@pytest.mark.parametrize("bcs", [(W.BC_ZERO, W.BC_PLANCK), (W.BC_PLANCK, W.BC_PLANCK)])
def test_linear_recording_reproduces_the_oracle_ray(oracle_mod, sgn, bcs):
    p = _column_problem(9, bcs[0], bcs[1], seed=3)
    rng = np.random.default_rng(4)
    i, j = 1, 2
    mu = float(sgn)
    for k0 in range(p.nz):
        S = 0.2 + rng.random(p.B.shape)
        ks, x = _ray(p, sgn, i, j, k0)
        c, TM = _linear_coefficients(oracle_mod, x)
        bc = bcs[0] if sgn > 0 else bcs[1]
        Ibc = p.B[ks[-1], j, i] if bc == W.BC_PLANCK else 0.0
        I = sum(c[m] * S[ks[m], j, i] for m in range(len(ks))) + TM * Ibc
        Io = oracle_mod.intensity(p, S, mu, 0.0, i, j, k0)
        assert I == pytest.approx(Io, rel=1e-13, abs=0)
        # the difference form replayed by the FP32 and double-float forms
        assert sum(c) + TM == pytest.approx(1.0, rel=0, abs=1e-14)
        S0 = S[ks[0], j, i]
        Id = sum(c[m] * (S[ks[m], j, i] - S0) for m in range(1, len(ks))) + TM * (Ibc - S0)
        assert Id + S0 == pytest.approx(Io, rel=1e-13, abs=0)


@pytest.mark.parametrize("sgn", [1, -1])
def test_parabolic_recording_reproduces_the_oracle_ray(oracle_mod, sgn):
    p = _column_problem(8, W.BC_PLANCK, W.BC_PLANCK, seed=5, src_order=1)
    rng = np.random.default_rng(6)
    i, j = 2, 0
    hs = p.dz / 2.0
    for k0 in range(p.nz):
        S = 0.2 + rng.random(p.B.shape)
        ks, x = _ray(p, sgn, i, j, k0)
        kd = k0 + sgn                       # the downstream point p_-1
        down = 0 <= kd < p.nz
        M = len(x)
        c = {}                              # point index (-1 .. M) -> coefficient
        T = 1.0
        xprev = hs * (p.chi[k0, j, i] + p.chi[kd, j, i]) if down else None
        for m in range(M):
            if m == 0 and not down:
                wc, wu = oracle_mod.weights(x[m])
                c[0] = c.get(0, 0.0) + wc
                c[1] = c.get(1, 0.0) + wu
            else:
                pu, pc, pd = oracle_mod.weights_parabolic(x[m], xprev)
                c[m + 1] = c.get(m + 1, 0.0) + T * pu
                c[m] = c.get(m, 0.0) + T * pc
                c[m - 1] = c.get(m - 1, 0.0) + T * pd
            T *= math.exp(-x[m])
            xprev = x[m]
        Ibc = p.B[ks[-1], j, i]
        I = T * Ibc
        for q, cq in c.items():
            kq = kd if q == -1 else ks[q]
            I += cq * S[kq, j, i]
        Io = oracle_mod.intensity(p, S, float(sgn), 0.0, i, j, k0)
        assert I == pytest.approx(Io, rel=1e-12, abs=0)


def test_truncated_recording_keeps_the_last_upwind_weight(oracle_mod):
    """A ray cut after L segments records c_L = T_{L-1} w_up,L-1 and no
    boundary term: the dropped tail is T_L times the rest of the ray."""
    p = _column_problem(12, W.BC_ZERO, W.BC_PLANCK, seed=7)
    S = np.ones(p.B.shape)
    ks, x = _ray(p, -1, 0, 0, 0)            # from the top plane down to the bottom
    L = 5
    c, TL = _linear_coefficients(oracle_mod, x[:L])
    assert c[L] == pytest.approx(np.prod([math.exp(-v) for v in x[:L - 1]])
                                 * oracle_mod.weights(x[L - 1])[1], rel=1e-14)
    # for S = 1 the full ray gives 1 - T_M + T_M B_bc; the cut one 1 - T_L
    assert sum(c) == pytest.approx(1.0 - TL, rel=0, abs=1e-14)
