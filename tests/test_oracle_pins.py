"""Pins of the FP64 oracle to facts that do not come from the oracle itself.

Each test checks the oracle against mathematics or physics that fix the
answer independently: high-precision evaluation of the segment weights,
closed-form intensities for pure absorption, exact numerical integration of
the linear-in-tau source along 1D rays, exact lattice geometry of single
characteristics, symmetries of the periodic slab, a brute-force Lambda
matrix (a full formal solution per unit source) and a direct dense solve of
the discrete scattering problem.  The paper (Hauschildt & Baron 2011)
prints no worked example, so these are the pins (Sect. 2.2, 2.3, 3.1).
"""

import math

import mpmath
import numpy as np
import pytest

from paper_1107_5719_gb300 import workloads as W

pytestmark = []


def _problem(nx, ny, nz, chi, S_or_B, mu, phi, w, eps=None, top=W.BC_ZERO,
             bottom=W.BC_PLANCK, dx=1.0, dy=1.0, dz=1.0):
    shape = (nz, ny, nx)
    chi = np.broadcast_to(np.asarray(chi, dtype=np.float64), shape).copy()
    B = np.broadcast_to(np.asarray(S_or_B, dtype=np.float64), shape).copy()
    eps = np.ones(shape) if eps is None else np.broadcast_to(np.asarray(eps, float), shape).copy()
    return W.Problem(nx, ny, nz, chi, eps, B, np.asarray(mu, float), np.asarray(phi, float),
                     np.asarray(w, float), dx=dx, dy=dy, dz=dz, top_bc=top, bottom_bc=bottom)


# ---------------------------------------------------------------- weights

def _weights_mp(x):
    x = mpmath.mpf(x)
    e = mpmath.exp(-x)
    q = -mpmath.expm1(-x) / x
    return 1 - q, q - e


@pytest.mark.parametrize("x", list(np.logspace(-12, 4, 97)) + [0.1 * (1 - 1e-15), 0.1, 0.5, 700.0])
def test_weights_match_high_precision(oracle_mod, x):
    """Segment weights against 40-digit evaluation of their definition."""
    mpmath.mp.dps = 40
    wc, wu = oracle_mod.weights(x)
    rc, ru = _weights_mp(x)
    assert abs(wc - float(rc)) <= 1e-14 * abs(float(rc))
    assert abs(wu - float(ru)) <= 1e-14 * abs(float(ru))


def test_weights_invariants_and_limits(oracle_mod):
    """w_cur + w_up = 1 - e^{-x}; both -> x/2 as x -> 0; w_cur -> 1 and
    w_up -> 1/x as x -> infinity; both are non-negative."""
    for x in np.logspace(-10, 3.5, 200):
        wc, wu = oracle_mod.weights(x)
        assert wc >= 0 and wu >= 0
        assert abs((wc + wu) - (-math.expm1(-x))) <= 4e-16 * max(1.0, -math.expm1(-x)) + 1e-16 * x
    wc, wu = oracle_mod.weights(1e-9)
    assert abs(wc / 5e-10 - 1) < 1e-8 and abs(wu / 5e-10 - 1) < 1e-8
    wc, wu = oracle_mod.weights(2000.0)
    assert abs(wc - (1 - 1 / 2000.0)) < 1e-15 and abs(wu - 1 / 2000.0) < 1e-15


# --------------------------------------------------- pure absorption pins

def test_pure_absorption_constant_chi_closed_form(oracle_mod):
    """Constant chi, S = B constant, eps = 1: every ray gives
    I = B (1 - e^{-tau}) + e^{-tau} I_bc with tau = chi M dz / |mu| (the
    linear-source scheme is exact for constant S)."""
    nx, ny, nz = 4, 3, 9
    chi, Bv = 0.37, 2.5
    mu, phi, w = W.quadrature(6, 5)
    p = _problem(nx, ny, nz, chi, Bv, mu, phi, w, dz=1.3, dx=0.7, dy=1.1)
    S = p.B.copy()
    J, _ = oracle_mod.formal_solution(p, S, lstar=False)
    for k in range(nz):
        Jref = 0.0
        for d in range(len(mu)):
            M = k if mu[d] > 0 else nz - 1 - k
            tau = chi * M * p.dz / abs(mu[d])
            Ibc = 0.0 if mu[d] > 0 else Bv
            Iref = Bv * (-math.expm1(-tau)) + math.exp(-tau) * Ibc
            I = oracle_mod.intensity(p, S, mu[d], phi[d], 1, 2, k)
            assert abs(I - Iref) <= 1e-14 * max(abs(Iref), 1e-300) + 1e-300
            Jref += w[d] * Iref
        assert np.allclose(J[k], Jref, rtol=1e-14, atol=0)


def test_pure_absorption_linear_chi_exact_tau(oracle_mod):
    """chi linear in depth: the trapezoid optical depth is exact, so
    I = B (1 - e^{-tau}) with tau the exact integral of chi along the ray."""
    nx, ny, nz = 3, 3, 12
    a, b = 0.05, 0.4
    k = np.arange(nz, dtype=float)
    chi = (a + b * k)[:, None, None]
    mu = np.array([0.83, -0.41, 0.17, -0.95])
    phi = np.array([0.3, 2.0, 4.0, 5.5])
    w = np.full(4, 0.25)
    p = _problem(nx, ny, nz, chi, 1.0, mu, phi, w, bottom=W.BC_ZERO, dz=0.8)
    S = p.B.copy()
    for k0 in range(nz):
        for d in range(4):
            kM = 0 if mu[d] > 0 else nz - 1
            lo, hi = sorted((k0, kM))
            tau = (p.dz / abs(mu[d])) * (a * (hi - lo) + b * (hi * hi - lo * lo) / 2.0)
            Iref = -math.expm1(-tau)
            I = oracle_mod.intensity(p, S, mu[d], phi[d], 2, 0, k0)
            assert abs(I - Iref) <= 2e-15 + 1e-14 * Iref


@pytest.mark.parametrize("variant", ["linear", "parabolic", "short"])
def test_diffusion_boundary_exact_for_linear_planck(oracle_mod, variant):
    _diffusion_pin(oracle_mod, variant)


def _diffusion_pin(oracle_mod, variant="linear"):
    """Pure absorption, constant chi, B linear in optical depth,
    B = a + c tau: the diffusion approximation I = B + |mu| dB/dtau is then
    the exact upward intensity, so with the LTE-diffusion inner boundary
    every upward ray at every depth gives B(tau_0) + |mu| c: the linear and
    the parabolic source integrate a linear source exactly, and the short
    characteristics interpolate a horizontally uniform plane exactly."""
    nx, ny, nz = 4, 3, 10
    chi, a, c, dz = 0.7, 2.0, 0.45, 1.3
    k = np.arange(nz, dtype=float)
    tau = chi * dz * k
    mu, phi, w = W.quadrature(8, 3)
    p = _problem(nx, ny, nz, chi, (a + c * tau)[:, None, None], mu, phi, w, dz=dz,
                 bottom=W.BC_DIFFUSION)
    p.src_order = 1 if variant == "parabolic" else 0
    S = p.B.copy()
    if variant == "short":
        # J from the upward directions only: zero weight on the downward ones
        up = mu < 0
        p.w = np.where(up, w, 0.0) / np.sum(w[up])
        J, _ = oracle_mod.formal_solution(p, S, lstar=False, method=oracle_mod.SHORT)
        ref = a + c * tau + np.sum(p.w * np.abs(mu)) * c
        assert np.allclose(J[:, 0, 0], ref, rtol=1e-13, atol=0)
        return
    for d in range(len(mu)):
        if mu[d] > 0:
            continue
        for k0 in range(nz):
            I = oracle_mod.intensity(p, S, mu[d], phi[d], 1, 2, k0)
            ref = a + c * tau[k0] + abs(mu[d]) * c
            assert abs(I - ref) <= 1e-13 * ref, (d, k0, I, ref)


# ------------------------------------- 1D rays with an exactly integrated source

def _ray_reference(chi_k, S_k, k0, mu, dz, Ibc):
    """Exact integral of S(t) e^{-t}, S linear in t between the nodes of a
    vertical-plane ray, nodes at trapezoid optical depths (40 digits)."""
    mpmath.mp.dps = 40
    nz = len(chi_k)
    s = 1 if mu > 0 else -1
    M = k0 if mu > 0 else nz - 1 - k0
    ds = mpmath.mpf(dz) / abs(mpmath.mpf(mu))
    t = [mpmath.mpf(0)]
    ks = [k0 - m * s for m in range(M + 1)]
    for m in range(M):
        t.append(t[-1] + ds * (mpmath.mpf(chi_k[ks[m]]) + mpmath.mpf(chi_k[ks[m + 1]])) / 2)
    I = mpmath.mpf(0)
    for m in range(M):
        t0, t1 = t[m], t[m + 1]
        s0, s1 = mpmath.mpf(S_k[ks[m]]), mpmath.mpf(S_k[ks[m + 1]])
        f = lambda tt: (s0 + (s1 - s0) * (tt - t0) / (t1 - t0)) * mpmath.exp(-tt)
        I += mpmath.quad(f, [t0, t1])
    I += mpmath.exp(-t[M]) * mpmath.mpf(Ibc)
    return float(I)


@pytest.mark.parametrize("method", [0, 1], ids=["long", "short"])
def test_horizontally_uniform_slab_equals_exact_1d_rays(oracle_mod, method):
    """Horizontally uniform chi and S: every (x,y) column gives the same J,
    equal to the exactly integrated 1D plane-parallel rays on the same
    z-grid and mu set (Sect. 3.1: the test slab is plane parallel).  Holds
    for long and short characteristics alike (interpolating a uniform plane
    is exact)."""
    nx, ny, nz = 5, 4, 13
    k = np.arange(nz, dtype=float)
    chi_k = 10.0 ** (-3.0 + 5.0 * k / (nz - 1))
    S_k = 1.0 + 0.5 * k / (nz - 1) + 0.3 * np.sin(1.7 * k)
    B_k = 1.0 + k / (nz - 1)
    mu, phi, w = W.quadrature(8, 3)
    p = _problem(nx, ny, nz, chi_k[:, None, None], B_k[:, None, None], mu, phi, w, dz=1.0)
    S = np.broadcast_to(S_k[:, None, None], (nz, ny, nx)).copy()
    J, _ = oracle_mod.formal_solution(p, S, lstar=False, method=method)
    assert np.max(np.abs(J - J[:, :1, :1])) <= 1e-14 * np.max(np.abs(J))
    for k0 in range(nz):
        Jref = 0.0
        for d in range(len(mu)):
            Ibc = 0.0 if mu[d] > 0 else B_k[-1]
            Jref += w[d] * _ray_reference(chi_k, S_k, k0, mu[d], p.dz, Ibc)
        assert abs(J[k0, 0, 0] - Jref) <= 1e-13 * abs(Jref), (k0, J[k0, 0, 0], Jref)


# ------------------------------------------------- lattice geometry pins

def _hat_reference(dtau, m, M):
    """Exact intensity from a unit source at node m of a ray with equal
    segments dtau (hat function in t), no boundary intensity."""
    mpmath.mp.dps = 40
    dt = mpmath.mpf(dtau)
    tm = m * dt
    total = mpmath.mpf(0)
    if m >= 1:
        total += mpmath.quad(lambda t: (t - (tm - dt)) / dt * mpmath.exp(-t), [tm - dt, tm])
    if m < M:
        total += mpmath.quad(lambda t: ((tm + dt) - t) / dt * mpmath.exp(-t), [tm, tm + dt])
    return float(total)


@pytest.mark.parametrize("mu_sign,phi,shift", [
    (+1, 0.0, (1, 0)),              # down-going, +x: upstream is -x, smaller k
    (-1, math.pi, (-1, 0)),         # up-going, -x: upstream is +x, larger k
    (+1, math.pi / 2, (0, 1)),      # +y
    (-1, 3 * math.pi / 2, (0, -1)),
])
def test_single_direction_unit_source_geometry(oracle_mod, mu_sign, phi, shift):
    """A direction at 45 degrees to the vertical in the x-z or y-z plane
    moves exactly one node sideways per plane.  A unit source at one node
    must light exactly the voxels downstream of it along the lattice line,
    with the exactly integrated hat-function intensity."""
    nx, ny, nz = 5, 6, 7
    chi = 0.6
    mu = mu_sign / math.sqrt(2.0)
    p = _problem(nx, ny, nz, chi, 0.0, [mu], [phi], [1.0], top=W.BC_ZERO, bottom=W.BC_ZERO)
    src = (1, 2, 3)  # (i, j, k)
    S = np.zeros((nz, ny, nx))
    S[src[2], src[1], src[0]] = 1.0
    dtau = chi * math.sqrt(2.0)
    sx, sy = shift
    s = 1 if mu > 0 else -1
    for k0 in range(nz):
        for j0 in range(ny):
            for i0 in range(nx):
                I = oracle_mod.intensity(p, S, mu, phi, i0, j0, k0)
                M = k0 if s > 0 else nz - 1 - k0
                m = (k0 - src[2]) * s
                expected = 0.0
                if 0 <= m <= M and (i0 - m * sx - src[0]) % nx == 0 and (j0 - m * sy - src[1]) % ny == 0:
                    expected = _hat_reference(dtau, m, M)
                assert abs(I - expected) <= 1e-13 * expected + 1e-14, (i0, j0, k0, I, expected)


def test_half_node_shift_splits_bilinearly(oracle_mod):
    """tan(theta) = 1/2 along +x: odd steps land half-way between nodes,
    so a unit source is seen with bilinear weight 1/2 by two voxels."""
    nx, ny, nz = 6, 3, 4
    mu = 2.0 / math.sqrt(5.0)
    p = _problem(nx, ny, nz, 1.0, 0.0, [mu], [0.0], [1.0], top=W.BC_ZERO, bottom=W.BC_ZERO)
    S = np.zeros((nz, ny, nx))
    S[0, 1, 2] = 1.0          # source in the top plane at x = 2
    # voxel (i0, *, k0=1): p_1 = i0 - 1/2.  x = 2 is a node of p_1 for i0 = 2 and 3
    I2 = oracle_mod.intensity(p, S, mu, 0.0, 2, 1, 1)
    I3 = oracle_mod.intensity(p, S, mu, 0.0, 3, 1, 1)
    I4 = oracle_mod.intensity(p, S, mu, 0.0, 4, 1, 1)
    dtau = 1.0 * 1.0 / mu
    full = _hat_reference(dtau, 1, 1)
    assert abs(I2 - 0.5 * full) < 1e-14 and abs(I3 - 0.5 * full) < 1e-14 and I4 == 0.0
    # voxel (i0, *, k0=2): p_2 = i0 - 1 hits x = 2 exactly for i0 = 3 only
    I3b = oracle_mod.intensity(p, S, mu, 0.0, 3, 1, 2)
    I2b = oracle_mod.intensity(p, S, mu, 0.0, 2, 1, 2)
    assert abs(I3b - _hat_reference(dtau, 2, 2)) < 1e-14 and abs(I2b) < 1e-15


# ------------------------------------------------------------ symmetries

def test_periodic_translation_invariance(oracle_mod):
    """Shifting every field by whole voxels in x and y (periodic wrap)
    shifts J and Lambda* by the same amount."""
    p = W.random_slab(5, 4, 6, n_theta=4, n_phi=6, seed=3)
    S = p.B * 0.7 + 0.1
    J, L = oracle_mod.formal_solution(p, S)
    sh = (2, 3)
    q = W.Problem(p.nx, p.ny, p.nz, np.roll(p.chi, sh, axis=(2, 1)), p.eps,
                  np.roll(p.B, sh, axis=(2, 1)), p.mu, p.phi, p.w)
    J2, L2 = oracle_mod.formal_solution(q, np.roll(S, sh, axis=(2, 1)))
    assert np.allclose(J2, np.roll(J, sh, axis=(2, 1)), rtol=1e-13, atol=0)
    assert np.allclose(L2, np.roll(L, sh, axis=(3, 2)), rtol=1e-13, atol=1e-300)


def test_mirror_symmetry(oracle_mod):
    """x -> -x maps the quadrature onto itself (phi -> pi - phi) and J onto
    the mirrored J; Lambda* offsets ox -> -ox."""
    p = W.random_slab(6, 5, 5, n_theta=4, n_phi=8, seed=5)
    S = p.B * 0.5 + 0.2
    J, L = oracle_mod.formal_solution(p, S)
    mir = lambda a: np.roll(a[..., ::-1], 1, axis=-1)     # i -> (nx - i) mod nx
    q = W.Problem(p.nx, p.ny, p.nz, mir(p.chi), p.eps, mir(p.B), p.mu, p.phi, p.w)
    J2, L2 = oracle_mod.formal_solution(q, mir(S))
    assert np.allclose(J2, mir(J), rtol=1e-13, atol=0)
    Lr = L.reshape(3, 3, 3, *L.shape[1:])[:, :, ::-1]      # ox -> -ox
    assert np.allclose(L2, mir(Lr.reshape(L.shape)), rtol=1e-12, atol=1e-300)


# ------------------------------------------------------ brute-force Lambda

def _brute_lambda(oracle_mod, p, method=0):
    N = p.nvox
    q = W.Problem(p.nx, p.ny, p.nz, p.chi, p.eps, p.B, p.mu, p.phi, p.w,
                  dx=p.dx, dy=p.dy, dz=p.dz, top_bc=W.BC_ZERO, bottom_bc=W.BC_ZERO,
                  src_order=p.src_order)
    Lam = np.empty((N, N))
    for j in range(N):
        S = np.zeros(N)
        S[j] = 1.0
        J, _ = oracle_mod.formal_solution(q, S.reshape(p.nz, p.ny, p.nx), lstar=False,
                                          method=method)
        Lam[:, j] = J.ravel()
    return Lam


def _neighbour(p, v, o):
    k, j, i = np.unravel_index(v, (p.nz, p.ny, p.nx))
    ox, oy, oz = o % 3 - 1, (o // 3) % 3 - 1, o // 9 - 1
    kk = k + oz
    if kk < 0 or kk >= p.nz:
        return -1
    return (kk * p.ny + (j + oy) % p.ny) * p.nx + (i + ox) % p.nx


@pytest.mark.parametrize("shape,seed", [((5, 5, 5), 11), ((3, 4, 5), 12)])
def test_lstar_at_equals_brute_force_lambda(oracle_mod, shape, seed):
    """Lambda* rows at a sample of voxels (the full-size spot-check call)
    equal the nearest-neighbour elements of the brute-force Lambda, for
    voxels listed in random order and with repeats (Sect. 2.2)."""
    nx, ny, nz = shape
    p = W.random_slab(nx, ny, nz, n_theta=4, n_phi=5, seed=seed)
    Lam = _brute_lambda(oracle_mod, p)
    rng = np.random.default_rng(seed)
    vox = np.concatenate([rng.permutation(p.nvox), rng.integers(0, p.nvox, 7)])
    rows = oracle_mod.lstar_at(p, vox)
    for q, v in enumerate(vox):
        for o in range(27):
            j = _neighbour(p, v, o)
            ref = 0.0 if j < 0 else Lam[v, j]
            assert abs(rows[q, o] - ref) <= 1e-14 * max(abs(ref), 1e-3), (v, o)


@pytest.mark.parametrize("shape,seed", [((5, 5, 5), 11), ((3, 4, 5), 12), ((4, 3, 2), 13)])
def test_lstar_equals_brute_force_lambda(oracle_mod, shape, seed):
    """Lambda* entries equal the matching elements of the full Lambda
    matrix built column by column from formal solutions with a unit source
    (Sect. 2.2: Lambda* is the nearest-neighbour part of Lambda)."""
    nx, ny, nz = shape
    p = W.random_slab(nx, ny, nz, n_theta=4, n_phi=5, seed=seed)
    S = p.B.copy()
    J, L = oracle_mod.formal_solution(p, S)
    Lam = _brute_lambda(oracle_mod, p)
    N = p.nvox
    Lf = L.reshape(27, N)
    for v in range(N):
        for o in range(27):
            j = _neighbour(p, v, o)
            if j < 0:
                assert Lf[o, v] == 0.0
            else:
                assert abs(Lf[o, v] - Lam[v, j]) <= 1e-14 * max(abs(Lam[v, j]), 1e-3), (v, o)
    # linearity: J(S) = Lambda S + J(S=0)
    rng = np.random.default_rng(seed)
    S2 = rng.random((nz, ny, nx)) * 3.0
    J2, _ = oracle_mod.formal_solution(p, S2, lstar=False)
    J0, _ = oracle_mod.formal_solution(p, np.zeros_like(S2), lstar=False)
    assert np.allclose(J2.ravel(), Lam @ S2.ravel() + J0.ravel(), rtol=1e-13, atol=1e-15)
    # positivity and row sums
    assert np.all(Lf >= 0.0)
    assert np.all(Lf.sum(axis=0) <= Lam.sum(axis=1) * (1 + 1e-14) + 1e-15)
    assert np.all(Lam.sum(axis=1) <= 1.0 + 1e-14)


# ------------------------------------------------------- parabolic source

def _parabolic_mp(a, b):
    """(P_up, P_cur, P_down) from 40-digit quadrature of the Lagrange basis
    through t = a, 0, -b against e^{-t} on [0, a]."""
    mpmath.mp.dps = 40
    a, b = mpmath.mpf(a), mpmath.mpf(b)
    Lu = lambda t: t * (t + b) / (a * (a + b))
    L0 = lambda t: (a - t) * (t + b) / (a * b)
    Ld = lambda t: t * (t - a) / (b * (a + b))
    return [float(mpmath.quad(lambda t: L(t) * mpmath.exp(-t), [0, a])) for L in (Lu, L0, Ld)]


@pytest.mark.parametrize("a", [1e-7, 3e-3, 0.2, 0.9999, 1.0, 2.5, 40.0, 800.0])
@pytest.mark.parametrize("b", [1e-6, 0.05, 1.0, 30.0])
def test_parabolic_weights_match_high_precision(oracle_mod, a, b):
    """Parabolic weights: 40-digit quadrature of each Lagrange basis
    polynomial against e^{-t}; they sum to 1 - e^{-a} and integrate t and t^2
    exactly."""
    w = oracle_mod.weights_parabolic(a, b)
    ref = _parabolic_mp(a, b)
    for x, r in zip(w, ref):
        assert abs(x - r) <= 1e-13 * abs(r) + 1e-300, (a, b, w, ref)
    E0 = -math.expm1(-a)
    assert abs(sum(w) - E0) <= 1e-14 * sum(abs(x) for x in w)


def test_parabolic_source_exact_for_quadratic_source(oracle_mod):
    """Horizontally uniform slab, chi rising with depth, pure absorption,
    zero boundaries, S quadratic in the (trapezoid) vertical optical depth
    tau: along every ray the optical depth is (tau - tau_0)/|mu|, so S is
    quadratic in it and the parabolic source integrates it exactly on
    unequal segments (all voxels with a downstream plane in both
    propagation senses, i.e. not the top and bottom planes), while the
    linear source does not."""
    nx, ny, nz = 4, 3, 9
    dz = 1.0
    k = np.arange(nz, dtype=float)
    chi_k = 0.2 * 10.0 ** (1.5 * k / (nz - 1))
    tau = np.concatenate([[0.0], np.cumsum(dz * (chi_k[1:] + chi_k[:-1]) / 2.0)])
    al, be, ga = 1.0, 0.8, 0.6
    S_k = al + be * tau + ga * tau ** 2
    mu, phi, w = W.quadrature(6, 2)
    p = _problem(nx, ny, nz, chi_k[:, None, None], S_k[:, None, None], mu, phi, w, dz=dz,
                 top=W.BC_ZERO, bottom=W.BC_ZERO)
    p.src_order = 1
    S = np.broadcast_to(S_k[:, None, None], (nz, ny, nx)).copy()
    mpmath.mp.dps = 30
    for k0 in range(1, nz - 1):
        for d in range(len(mu)):
            amu = abs(mu[d])
            tb = tau[0] if mu[d] > 0 else tau[-1]       # depth of the entry plane
            t_M = abs(tau[k0] - tb) / amu
            sgn = 1.0 if mu[d] > 0 else -1.0
            # along the ray t = |tau0 - tau| / |mu|: tau = tau0 - sgn |mu| t
            f = lambda t: (al + be * (tau[k0] - sgn * amu * t) + ga * (tau[k0] - sgn * amu * t) ** 2) \
                * mpmath.exp(-t)
            ref = float(mpmath.quad(f, [0, t_M]))
            I = oracle_mod.intensity(p, S, mu[d], phi[d], 1, 1, k0)
            assert abs(I - ref) <= 1e-13 * ref, (k0, d, I, ref)
    p.src_order = 0
    I_lin = oracle_mod.intensity(p, S, mu[0], phi[0], 1, 1, nz // 2)
    p.src_order = 1
    I_par = oracle_mod.intensity(p, S, mu[0], phi[0], 1, 1, nz // 2)
    assert abs(I_lin - I_par) > 1e-6 * abs(I_par)


@pytest.mark.parametrize("shape,seed", [((4, 4, 4), 16), ((3, 5, 4), 17)])
def test_parabolic_lstar_equals_brute_force_lambda(oracle_mod, shape, seed):
    """The parabolic-source Lambda* equals the matching elements of its full
    Lambda (unit-source formal solutions), including the downstream plane."""
    nx, ny, nz = shape
    p = W.random_slab(nx, ny, nz, n_theta=4, n_phi=5, seed=seed)
    p.src_order = 1
    J, L = oracle_mod.formal_solution(p, p.B)
    q = W.Problem(p.nx, p.ny, p.nz, p.chi, p.eps, p.B, p.mu, p.phi, p.w, src_order=1,
                  top_bc=W.BC_ZERO, bottom_bc=W.BC_ZERO)
    Lam = _brute_lambda(oracle_mod, q)
    N = p.nvox
    Lf = L.reshape(27, N)
    for v in range(N):
        for o in range(27):
            j = _neighbour(p, v, o)
            if j < 0:
                assert Lf[o, v] == 0.0
            else:
                assert abs(Lf[o, v] - Lam[v, j]) <= 1e-14 * max(abs(Lam[v, j]), 1e-3), (v, o)
    # the downstream plane carries entries (negative ones among them)
    assert np.any(Lf[18:] != 0.0) and np.any(Lf[:9] != 0.0) and np.any(Lf < 0.0)


# ------------------------------------------------- short characteristics

def _lattice_direction_problem(top, bottom):
    """Directions whose per-plane shift (ax, ay) is a lattice vector, so that
    the upstream point of every node is itself a node."""
    p = W.random_slab(7, 6, 8, n_theta=2, n_phi=1, seed=5, top_bc=top, bottom_bc=bottom)
    r2, r3, r5 = math.sqrt(2.0), math.sqrt(3.0), math.sqrt(5.0)
    p.mu = np.array([1 / r2, -1 / r2, 1 / r3, -1 / r5, 1.0, -1 / r2, -1 / r3])
    p.phi = np.array([0.0, math.pi / 2, math.pi / 4, math.pi, 0.3, 1.5 * math.pi,
                      1.25 * math.pi])
    p.w = np.full(7, 1.0 / 7.0)
    return p


@pytest.mark.parametrize("bc", [(0, 1), (1, 0), (0, 2)])
def test_short_characteristics_equal_long_on_lattice_directions(oracle_mod, bc):
    """When every upstream point is a lattice node, interpolating the
    intensity there is exact, so the short-characteristics J and Lambda*
    equal the long-characteristics ones for arbitrary 3D chi and S."""
    p = _lattice_direction_problem(*bc)
    S = 0.5 + np.random.default_rng(1).random(p.B.shape)
    Jl, Ll = oracle_mod.formal_solution(p, S)
    Js, Ls = oracle_mod.formal_solution(p, S, method=oracle_mod.SHORT)
    assert np.allclose(Js, Jl, rtol=1e-13, atol=0)
    assert np.max(np.abs(Ls - Ll)) <= 1e-14


@pytest.mark.parametrize("shape,seed", [((4, 4, 4), 14), ((3, 5, 4), 15)])
def test_short_lstar_equals_brute_force_lambda(oracle_mod, shape, seed):
    """The short-characteristics Lambda* equals the matching elements of its
    full Lambda, built column by column from unit-source formal solutions;
    J is linear in S with that Lambda."""
    nx, ny, nz = shape
    p = W.random_slab(nx, ny, nz, n_theta=4, n_phi=5, seed=seed)
    J, L = oracle_mod.formal_solution(p, p.B, method=oracle_mod.SHORT)
    Lam = _brute_lambda(oracle_mod, p, method=oracle_mod.SHORT)
    N = p.nvox
    Lf = L.reshape(27, N)
    for v in range(N):
        for o in range(27):
            j = _neighbour(p, v, o)
            if j < 0:
                assert Lf[o, v] == 0.0
            else:
                assert abs(Lf[o, v] - Lam[v, j]) <= 1e-14 * max(abs(Lam[v, j]), 1e-3), (v, o)
    rng = np.random.default_rng(seed)
    S2 = rng.random((nz, ny, nx)) * 3.0
    J2, _ = oracle_mod.formal_solution(p, S2, lstar=False, method=oracle_mod.SHORT)
    J0, _ = oracle_mod.formal_solution(p, np.zeros_like(S2), lstar=False,
                                       method=oracle_mod.SHORT)
    assert np.allclose(J2.ravel(), Lam @ S2.ravel() + J0.ravel(), rtol=1e-13, atol=1e-15)
    assert np.all(Lf >= 0.0) and np.all(Lam.sum(axis=1) <= 1.0 + 1e-14)


def test_short_characteristics_converged_ali_equals_dense_solution(oracle_mod):
    """Outer iteration with the short-characteristics formal solution: the
    fixed point J = Lambda_sc (eps B + (1 - eps) J) + J_bc, solved directly."""
    p = W.random_slab(5, 5, 5, n_theta=4, n_phi=5, seed=31, eps_range=(1e-2, 1.0))
    r = oracle_mod.solve(p, tol=1e-14, max_iter=400, tol_inner=1e-14, max_sweeps=2000,
                         fs_method=oracle_mod.SHORT)
    assert r["converged"]
    Lam = _brute_lambda(oracle_mod, p, method=oracle_mod.SHORT)
    J0, _ = oracle_mod.formal_solution(p, np.zeros_like(p.B), lstar=False,
                                       method=oracle_mod.SHORT)
    eps = p.eps.ravel()
    A = np.eye(p.nvox) - Lam * (1 - eps)[None, :]
    ref = np.linalg.solve(A, Lam @ (eps * p.B.ravel()) + J0.ravel())
    assert np.allclose(r["J"].ravel(), ref, rtol=1e-11, atol=0)


# ------------------------------------------- operator splitting and ALI

def _dense_lstar(p, L):
    N = p.nvox
    A = np.zeros((N, N))
    Lf = L.reshape(27, N)
    for v in range(N):
        for o in range(27):
            j = _neighbour(p, v, o)
            if j >= 0:
                A[v, j] += Lf[o, v]
    return A


def test_os_step_solves_its_linear_system(oracle_mod):
    """Jacobi sweeps to a tight tolerance reproduce the direct solution of
    (1 - Lambda* D) J_new = J_fs - Lambda* D J_old (Sect. 2.3)."""
    p = W.random_slab(4, 5, 6, n_theta=4, n_phi=4, seed=21, eps_range=(1e-3, 1.0))
    S = p.eps * p.B + (1 - p.eps) * p.B
    Jfs, L = oracle_mod.formal_solution(p, S)
    rng = np.random.default_rng(1)
    Jold = p.B * (0.5 + rng.random(p.B.shape))
    Jn, ns = oracle_mod.os_step(p, L, Jfs, Jold, tol_inner=1e-15, max_sweeps=5000)
    A = _dense_lstar(p, L)
    Dg = np.diag(1 - p.eps.ravel())
    lhs = np.eye(p.nvox) - A @ Dg
    rhs = Jfs.ravel() - A @ Dg @ Jold.ravel()
    ref = np.linalg.solve(lhs, rhs)
    assert ns > 1
    assert np.allclose(Jn.ravel(), ref, rtol=1e-12, atol=0)


def _os_dense(p, L, Jfs, Jold):
    """(M, b) of the operator-splitting system M J_new = b in dense form."""
    A = _dense_lstar(p, L)
    Dg = np.diag(1 - p.eps.ravel())
    return np.eye(p.nvox) - A @ Dg, Jfs.ravel() - A @ Dg @ Jold.ravel()


def test_gauss_seidel_solves_its_linear_system(oracle_mod):
    """Red-black Gauss-Seidel sweeps reach the same direct solution as the
    Jacobi sweeps (Sect. 2.3), in fewer sweeps: the matrix 1 - Lambda* D is
    an M-matrix (Lambda* >= 0, row sums < 1), for which the splitting that
    takes the new values of the other colour converges at least as fast."""
    p = W.random_slab(4, 5, 6, n_theta=4, n_phi=4, seed=21, eps_range=(1e-3, 1.0))
    S = p.eps * p.B + (1 - p.eps) * p.B
    Jfs, L = oracle_mod.formal_solution(p, S)
    rng = np.random.default_rng(1)
    Jold = p.B * (0.5 + rng.random(p.B.shape))
    M, b = _os_dense(p, L, Jfs, Jold)
    ref = np.linalg.solve(M, b)
    Jj, nj = oracle_mod.os_step(p, L, Jfs, Jold, tol_inner=1e-14, max_sweeps=5000)
    Jg, ng = oracle_mod.os_step(p, L, Jfs, Jold, tol_inner=1e-14, max_sweeps=5000,
                                method=oracle_mod.GAUSS_SEIDEL)
    assert np.allclose(Jg.ravel(), ref, rtol=1e-12, atol=0)
    assert np.allclose(Jj.ravel(), ref, rtol=1e-12, atol=0)
    assert 1 < ng < nj


@pytest.mark.parametrize("shape,seed", [((4, 4, 3), 3), ((3, 5, 4), 4)])
def test_gauss_seidel_sweep_equals_block_form(oracle_mod, shape, seed):
    """One red-black sweep in the textbook block form: order the unknowns
    red (i+j+k even) then black, split M = Dm - C (Dm its diagonal); then
    x_r' = Dm_r^-1 (b_r + C_rr x_r + C_rb x_b),
    x_b' = Dm_b^-1 (b_b + C_br x_r' + C_bb x_b).  Synthetic positive Lambda*
    on all 27 offsets; shape (3, 5, 4) has odd periods, where equal colours
    meet across the seam."""
    nx, ny, nz = shape
    p = W.random_slab(nx, ny, nz, n_theta=2, n_phi=1, seed=seed, eps_range=(1e-2, 1.0))
    rng = np.random.default_rng(seed)
    L = rng.random((27, nz, ny, nx)) * 0.03
    L[:9, 0] = 0.0        # no plane above the top
    L[18:, -1] = 0.0      # no plane below the bottom
    Jfs = 1 + rng.random((nz, ny, nx))
    Jold = 1 + rng.random((nz, ny, nx))
    M, b = _os_dense(p, L, Jfs, Jold)
    Dm = np.diag(M).copy()
    Cm = np.diag(Dm) - M
    kk, jj, ii = np.unravel_index(np.arange(p.nvox), (nz, ny, nx))
    red = (ii + jj + kk) % 2 == 0
    blk = ~red
    x = Jold.ravel().copy()
    xr = (b[red] + Cm[np.ix_(red, red)] @ x[red] + Cm[np.ix_(red, blk)] @ x[blk]) / Dm[red]
    xb = (b[blk] + Cm[np.ix_(blk, red)] @ xr + Cm[np.ix_(blk, blk)] @ x[blk]) / Dm[blk]
    ref = np.empty(p.nvox)
    ref[red], ref[blk] = xr, xb
    Jg, ns = oracle_mod.os_step(p, L, Jfs, Jold, tol_inner=0.0, max_sweeps=1,
                                method=oracle_mod.GAUSS_SEIDEL)
    assert ns == 1
    assert np.allclose(Jg.ravel(), ref, rtol=1e-14, atol=0)
    # the Jacobi sweep is the same block form with x_r' replaced by x_r
    xbj = (b[blk] + Cm[np.ix_(blk, red)] @ x[red] + Cm[np.ix_(blk, blk)] @ x[blk]) / Dm[blk]
    Jj, _ = oracle_mod.os_step(p, L, Jfs, Jold, tol_inner=0.0, max_sweeps=1)
    assert np.allclose(Jj.ravel()[blk], xbj, rtol=1e-14, atol=0)
    assert np.allclose(Jj.ravel()[red], xr, rtol=1e-14, atol=0)


def test_gauss_seidel_ali_reaches_the_same_fixed_point(oracle_mod):
    """The outer iteration with Gauss-Seidel operator splitting converges to
    the same J as with Jacobi sweeps, with fewer inner sweeps."""
    p = W.random_slab(5, 5, 5, n_theta=4, n_phi=5, seed=31, eps_range=(1e-2, 1.0))
    rj = oracle_mod.solve(p, tol=1e-13, max_iter=400, tol_inner=1e-13, max_sweeps=2000)
    rg = oracle_mod.solve(p, tol=1e-13, max_iter=400, tol_inner=1e-13, max_sweeps=2000,
                          os_method=oracle_mod.GAUSS_SEIDEL)
    assert rj["converged"] and rg["converged"]
    assert np.allclose(rg["J"], rj["J"], rtol=1e-11, atol=0)
    assert rg["sweeps"].sum() < rj["sweeps"].sum()


def test_converged_ali_equals_dense_solution(oracle_mod):
    """The converged outer iteration is the unique fixed point
    J = Lambda (eps B + (1 - eps) J) + J_bc, solved directly with the
    brute-force Lambda (Sect. 2, Sect. 3.1 item 5)."""
    p = W.random_slab(5, 5, 5, n_theta=4, n_phi=5, seed=31, eps_range=(1e-2, 1.0))
    r = oracle_mod.solve(p, tol=1e-14, max_iter=400, tol_inner=1e-14, max_sweeps=2000)
    assert r["converged"]
    Lam = _brute_lambda(oracle_mod, p)
    J0, _ = oracle_mod.formal_solution(p, np.zeros_like(p.B), lstar=False)
    eps = p.eps.ravel()
    A = np.eye(p.nvox) - Lam * (1 - eps)[None, :]
    ref = np.linalg.solve(A, Lam @ (eps * p.B.ravel()) + J0.ravel())
    assert np.allclose(r["J"].ravel(), ref, rtol=1e-11, atol=0)


def test_ng_extrapolation_exact_for_two_geometric_modes(oracle_mod):
    """If the error of the iterates is a sum of two geometric modes,
    x_k = x* + A l1^k + C l2^k, second-order Ng extrapolation of the four
    latest iterates returns x* exactly (the polynomial with roots l1, l2
    annihilates both modes)."""
    rng = np.random.default_rng(4)
    n = 200
    xs = 1.0 + rng.random(n)
    A, Cm = rng.standard_normal(n), rng.standard_normal(n)
    for l1, l2 in ((0.9, 0.5), (0.99, -0.3), (0.95, 0.8), (-0.7, 0.6)):
        it = [xs + A * l1 ** k + Cm * l2 ** k for k in range(6)]
        x, a, b, sing = oracle_mod.ng_step(it[5], it[4], it[3], it[2])
        assert not sing
        # coefficients of the polynomial with roots l1, l2 normalised to p(1) = 1
        den = (1 - l1) * (1 - l2)
        assert abs(a - (-(l1 + l2) / den)) < 1e-7 * abs(a)
        assert abs(b - (l1 * l2 / den)) < 1e-7 * abs(b)
        # the plain iterate is off by ~l1^5; the extrapolation by rounding only
        assert np.max(np.abs(x - xs) / xs) < 1e-8, (l1, l2)
        assert np.max(np.abs(it[5] - xs) / xs) > 1e-3


def test_ng_accelerated_ali_reaches_the_same_fixed_point(oracle_mod):
    p = W.random_slab(5, 5, 5, n_theta=4, n_phi=5, seed=31, eps_range=(1e-3, 1.0))
    plain = oracle_mod.solve(p, tol=1e-13, max_iter=2000, tol_inner=1e-14, max_sweeps=2000)
    ng = oracle_mod.solve(p, tol=1e-13, max_iter=2000, tol_inner=1e-14, max_sweeps=2000,
                          ng_period=4)
    assert plain["converged"] and ng["converged"]
    assert ng["iters"] < plain["iters"]
    assert np.allclose(ng["J"], plain["J"], rtol=1e-10, atol=0)


def test_ng_threshold_switches_extrapolation_off(oracle_mod):
    """With a minimum delta above every delta of the run, Ng never
    extrapolates and the iteration is exactly the plain one."""
    p = W.random_slab(5, 4, 6, n_theta=4, n_phi=4, seed=8, eps_range=(1e-2, 1.0))
    plain = oracle_mod.solve(p, tol=1e-10, max_iter=500, tol_inner=0.0, max_sweeps=10)
    off = oracle_mod.solve(p, tol=1e-10, max_iter=500, tol_inner=0.0, max_sweeps=10,
                           ng_period=4, ng_min_delta=1e30)
    assert off["iters"] == plain["iters"]
    assert np.array_equal(off["J"], plain["J"])
    on = oracle_mod.solve(p, tol=1e-10, max_iter=500, tol_inner=0.0, max_sweeps=10,
                          ng_period=4, ng_min_delta=1e-6)
    assert on["iters"] < plain["iters"]
    assert np.allclose(on["J"], plain["J"], rtol=1e-8, atol=0)


# ------------------------------------------------------------- physics

def test_thermalisation_at_depth(oracle_mod):
    """Deep in the slab (optical depth >> 1/sqrt(eps)) J -> B."""
    p = W.slab_small(n_theta=8, n_phi=4)
    r = oracle_mod.solve(p, max_iter=300)
    assert r["converged"]
    J = r["J"]
    dev = [np.max(np.abs(J[k] / p.B[k] - 1.0)) for k in range(p.nz // 2, p.nz)]
    assert all(a > b for a, b in zip(dev, dev[1:]))          # monotone approach
    assert dev[-3] < 1e-3 and dev[-1] < 1e-8
    assert np.all(J > 0) and np.all(J <= p.B * (1 + 1e-12))


def _surface_source(oracle_mod, nz, eps, decades=9.0):
    k = np.arange(nz, dtype=float)
    tau = 1e-5 * 10.0 ** (decades * k / (nz - 1))
    chi = np.gradient(tau)
    mu, phi, w = W.quadrature(8, 1)
    p = _problem(3, 3, nz, chi[:, None, None], 1.0, mu, phi, w, eps=eps)
    r = oracle_mod.solve(p, tol=1e-10, max_iter=3000, tol_inner=1e-13, max_sweeps=3000)
    assert r["converged"]
    return eps + (1 - eps) * r["J"][0, 0, 0]


def test_sqrt_eps_surface_law(oracle_mod):
    """Semi-infinite isothermal scattering atmosphere: S(0) = sqrt(eps) B.
    Horizontally uniform 3x3 columns on logarithmic depth grids spanning
    nine decades; the error must shrink under refinement and be within 5%
    on the 121-plane grid (measured: 0.902, 0.965, 0.989 of sqrt(eps) for
    61, 121, 241 planes)."""
    eps = 1e-2
    s61 = _surface_source(oracle_mod, 61, eps) / math.sqrt(eps)
    s121 = _surface_source(oracle_mod, 121, eps) / math.sqrt(eps)
    assert abs(s121 - 1.0) < 0.05, s121
    assert abs(s121 - 1.0) < 0.5 * abs(s61 - 1.0), (s61, s121)


# ----------------------------------------------------------- quadrature

@pytest.mark.parametrize("nt,nphi", [(2, 1), (8, 3), (16, 16), (64, 64)])
def test_quadrature_moments(nt, nphi):
    """sum w = 1; sum w mu^{2k} = 1/(2k+1) for 2k <= 2 n_theta - 1; odd
    moments vanish; azimuthal moments sum w cos(phi) = sum w sin(phi) = 0."""
    mu, phi, w = W.quadrature(nt, nphi)
    assert abs(w.sum() - 1.0) < 1e-14
    for kk in range(0, nt):
        assert abs(np.sum(w * mu ** (2 * kk)) - 1.0 / (2 * kk + 1)) < 1e-13
        assert abs(np.sum(w * mu ** (2 * kk + 1))) < 1e-14
    assert np.all(np.abs(mu) > 0)
    if nphi > 1:
        assert abs(np.sum(w * np.cos(phi))) < 1e-14 and abs(np.sum(w * np.sin(phi))) < 1e-14


# ------------------------------------------------------ planted mistakes

_MUTANTS = {
    "swap_segment_weights": ("*w_cur = 1.0 - one_minus_e / x;\n        *w_up = one_minus_e / x - e;",
                             "*w_up = 1.0 - one_minus_e / x;\n        *w_cur = one_minus_e / x - e;"),
    "taylor_sign": ("double sgn = (n % 2) ? 1.0 : -1.0;", "double sgn = 1.0;"),
    "left_point_dtau": ("double dtau = d.ds * (chi_a + chi_b) / 2.0;", "double dtau = d.ds * chi_a;"),
    "upstream_sign_x": ("d.ax = (g->dz / g->dx) * sint * cos(phi) / amu;",
                        "d.ax = -(g->dz / g->dx) * sint * cos(phi) / amu;"),
    "path_length_mu": ("d.ds = g->dz / amu;", "d.ds = g->dz * amu;"),
    "steps_off_by_one": ("return d->s > 0 ? (int)k0 : (int)(g->nz - 1 - k0);",
                         "return d->s > 0 ? (int)k0 : (int)(g->nz - 2 - k0);"),
    "no_boundary_intensity": ("double I = bc ? bilinear(g, B, kM, xM, yM) : 0.0;", "double I = 0.0;"),
    "bilinear_transposed": ("+ tx * (1.0 - ty) * f[vidx(g, i1, j0, k)]\n         + (1.0 - tx) * ty * f[vidx(g, i0, j1, k)]",
                            "+ ty * (1.0 - tx) * f[vidx(g, i1, j0, k)]\n         + (1.0 - ty) * tx * f[vidx(g, i0, j1, k)]"),
    "lstar_xy_swapped": ("return ((int)dzv + 1) * 9 + (oy + 1) * 3 + (ox + 1);",
                         "return ((int)dzv + 1) * 9 + (ox + 1) * 3 + (oy + 1);"),
    "lstar_drops_upstream_term": ("if (m >= 1) c += T[m - 1] * wu[m - 1];", "(void)0;"),
    "lstar_at_rows_reversed": ("double *row = lstar_out + q * 27;",
                               "double *row = lstar_out + (nsample - 1 - q) * 27;"),
    "os_forgets_destruction": ("r -= lstar[(long)o * N + v] * (1.0 - eps[j]) * J_old[j];",
                               "r -= lstar[(long)o * N + v] * J_old[j];"),
    "os_diag_uses_neighbour_eps": ("return acc / (1.0 - lstar[13L * N + v] * (1.0 - eps[v]));",
                                   "return acc / (1.0 - lstar[13L * N + v]);"),
    "parabolic_up_down_swapped": ("*p_up = (E[2] + b * E[1]) / (a * (a + b));",
                                  "*p_up = (E[2] - a * E[1]) / (b * (a + b));"),
    "parabolic_downstream_depth_from_upstream": ("orc_weights_parabolic(dtau[m + 1], dtau[m], wu, wc, wd);",
                                                 "orc_weights_parabolic(dtau[m + 1], dtau[m + 1], wu, wc, wd);"),
    "parabolic_lstar_drops_downstream": ("if (j + 1 < M) c += T[j + 1] * wdn[j + 1];", "(void)0;"),
    "sc_upstream_on_own_plane": ("long ku = k - d.s;\n                double x = (double)i - d.ax",
                                 "long ku = k;\n                double x = (double)i - d.ax"),
    "sc_no_attenuation": ("I[v] = bilinear(g, I, ku, x, y) * e + wc * S[v]",
                          "I[v] = bilinear(g, I, ku, x, y) + wc * S[v]"),
    "sc_lstar_drops_corner_segment": ("if (o >= 0) lrow[o] += wd * bx[a] * by[b] * (wu + e * wcc);",
                                      "if (o >= 0) lrow[o] += wd * bx[a] * by[b] * wu;"),
    "gs_black_uses_old_red": ("upd[v] = os_update(g, lstar, eps, rhs, Jn, v, N);",
                              "upd[v] = os_update(g, lstar, eps, rhs, Jc, v, N);"),
    "gs_colour_ignores_depth": ("return (int)((i + j + k) & 1);", "return (int)((i + j) & 1);"),
    "gs_sequential_within_colour": ("if (colour_of(g, v) == colour) upd[v] = os_update(g, lstar, eps, rhs, Jn, v, N);",
                                    "if (colour_of(g, v) == colour) Jn[v] = upd[v] = os_update(g, lstar, eps, rhs, Jn, v, N);"),
    "source_function_sign": ("S[v] = eps[v] * B[v] + (1.0 - eps[v]) * J[v];",
                             "S[v] = eps[v] * J[v] + (1.0 - eps[v]) * B[v];"),
    "ng_coefficients_swapped": ("for (long i = 0; i < N; ++i) out[i] = (1.0 - a - b) * x0[i] + a * x1[i] + b * x2[i];",
                                "for (long i = 0; i < N; ++i) out[i] = (1.0 - a - b) * x0[i] + b * x1[i] + a * x2[i];"),
    "ng_unweighted_cross_term": ("a12 += w * q1 * q2;", "a12 += q1 * q2;"),
    "diffusion_without_mu": ("if (bc == 2) I += fabs(mu) * diffusion_gradient_at(g, chi, B, xM, yM);",
                             "if (bc == 2) I += diffusion_gradient_at(g, chi, B, xM, yM);"),
    "diffusion_gradient_sign": ("long a = vidx(g, i, j, g->nz - 1), b = vidx(g, i, j, g->nz - 2);",
                                "long b = vidx(g, i, j, g->nz - 1), a = vidx(g, i, j, g->nz - 2);"),
}


def _pin_battery(mod):
    """Cheap pins first; returns the name of the first pin that fails."""
    pins = [
        ("weights", lambda: [test_weights_match_high_precision(mod, x) for x in (1e-3, 0.05, 0.3, 3.0, 40.0)]),
        ("absorption", lambda: test_pure_absorption_constant_chi_closed_form(mod)),
        ("linear_chi", lambda: test_pure_absorption_linear_chi_exact_tau(mod)),
        ("geometry", lambda: test_single_direction_unit_source_geometry(mod, +1, 0.0, (1, 0))),
        ("half_node", lambda: test_half_node_shift_splits_bilinearly(mod)),
        ("lstar", lambda: test_lstar_equals_brute_force_lambda(mod, (3, 4, 5), 12)),
        ("lstar_at", lambda: test_lstar_at_equals_brute_force_lambda(mod, (3, 4, 5), 12)),
        ("short", lambda: test_short_characteristics_equal_long_on_lattice_directions(mod, (0, 1))),
        ("parabolic", lambda: test_parabolic_weights_match_high_precision(mod, 0.2, 0.05)),
        ("parabolic_exact", lambda: test_parabolic_source_exact_for_quadratic_source(mod)),
        ("parabolic_lstar", lambda: test_parabolic_lstar_equals_brute_force_lambda(mod, (3, 5, 4), 17)),
        ("short_lstar", lambda: test_short_lstar_equals_brute_force_lambda(mod, (3, 5, 4), 15)),
        ("os_step", lambda: test_os_step_solves_its_linear_system(mod)),
        ("gauss_seidel", lambda: test_gauss_seidel_sweep_equals_block_form(mod, (3, 5, 4), 4)),
        ("ali", lambda: test_converged_ali_equals_dense_solution(mod)),
        ("ng", lambda: test_ng_extrapolation_exact_for_two_geometric_modes(mod)),
        ("diffusion", lambda: _diffusion_pin(mod)),
    ]
    for name, fn in pins:
        try:
            fn()
        except AssertionError:
            return name
    return None


@pytest.mark.parametrize("mutant", sorted(_MUTANTS))
def test_planted_mistake_is_caught(oracle_mod, mutant, tmp_path, monkeypatch):
    """Each plausible mistake planted in a copy of the oracle's source makes
    at least one pin fail; the unmodified oracle passes them all."""
    import ctypes
    import subprocess
    old, new = _MUTANTS[mutant]
    src = open(oracle_mod._SRC).read()
    assert src.count(old) == 1, mutant
    path = tmp_path / "mutant.c"
    path.write_text(src.replace(old, new))
    so = tmp_path / "libmutant.so"
    subprocess.run(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-fopenmp",
                    "-ffp-contract=off", "-o", str(so), str(path), "-lm"], check=True)
    lib = oracle_mod._configure(ctypes.CDLL(str(so)))
    monkeypatch.setattr(oracle_mod, "_lib", lib)
    assert _pin_battery(oracle_mod) is not None, f"mutant {mutant} passed every pin"


def test_unmodified_oracle_passes_pin_battery(oracle_mod):
    assert _pin_battery(oracle_mod) is None
