"""Seeded synthetic inputs for the 3DRT hot path.

This module only draws inputs: grids, opacities chi, thermalisation
parameters eps, Planck functions B, boundary modes and the solid-angle
quadrature. It contains none of the method's arithmetic (no formal
solution, no Lambda*, no operator splitting), so both the CUDA path and the
oracle can be fed from it without sharing any computation.

The slabs imitate the paper's continuum test model (Sect. 3.1): a plane
parallel slab, periodic in x and y, the outer boundary at the top (depth
index k = 0, incoming intensity zero) and the inner boundary at the bottom
(k = nz - 1, incoming intensity B), a grey opacity that rises as a power of
ten with depth so that the optical depth spans many decades, and coherent
isotropic scattering with thermalisation parameter eps (Sect. 3.1, list
item 5). The paper does not give its depth grid, its direction set or the
horizontal structure, so the laws below are the synthetic stand-ins; every
array is drawn with numpy's ``default_rng`` from a stated seed.

Arrays are C-ordered [nz][ny][nx] (x fastest), float64.
"""

from __future__ import annotations

import dataclasses
import math
from typing import List, Optional

import numpy as np

BC_ZERO = 0     # incoming intensity 0 (outer boundary, Sect. 3.1 item 4)
BC_PLANCK = 1   # incoming intensity B at the entry point (inner boundary)
BC_DIFFUSION = 2  # inner boundary only: B + |mu| dB/dtau (LTE diffusion, Sect. 3.1 item 4)

SEED_BASE = 1234


@dataclasses.dataclass
class Problem:
    """One monochromatic 3DRT problem on an x/y periodic slab."""

    nx: int
    ny: int
    nz: int
    chi: np.ndarray
    eps: np.ndarray
    B: np.ndarray
    mu: np.ndarray
    phi: np.ndarray
    w: np.ndarray
    dx: float = 1.0
    dy: float = 1.0
    dz: float = 1.0
    top_bc: int = BC_ZERO
    bottom_bc: int = BC_PLANCK
    tol: float = 1e-8
    name: str = ""
    src_order: int = 0      # 0: linear source on each segment, 1: parabolic

    @property
    def nvox(self) -> int:
        return self.nx * self.ny * self.nz

    @property
    def ndir(self) -> int:
        return int(self.mu.shape[0])


def quadrature(n_theta: int, n_phi: int):
    """Product quadrature over the unit sphere.

    mu: full-range Gauss-Legendre nodes on [-1, 1] (n_theta even, so no
    node has mu = 0); phi_l = 2 pi (l + 1/2) / n_phi, offset by half a step
    so that no direction is aligned with an axis or a diagonal; weights
    w = (a_m / 2) / n_phi so that sum(w) = 1 and J = sum_d w_d I_d.
    Directions are ordered mu-major, phi-minor.
    """
    if n_theta < 2 or n_theta % 2:
        raise ValueError("n_theta must be even and >= 2")
    if n_phi < 1:
        raise ValueError("n_phi must be >= 1")
    x, a = np.polynomial.legendre.leggauss(n_theta)
    phis = 2.0 * math.pi * (np.arange(n_phi) + 0.5) / n_phi
    mu = np.repeat(x, n_phi)
    phi = np.tile(phis, n_theta)
    w = np.repeat(a / 2.0, n_phi) / n_phi
    return mu.astype(np.float64), phi.astype(np.float64), w.astype(np.float64)


def _depth(nz: int) -> np.ndarray:
    return np.arange(nz, dtype=np.float64)[:, None, None]


def slab_small(uniform: bool = False, eps: float = 1e-2, n_theta: int = 16,
               n_phi: int = 16, n: int = 17, seed: Optional[int] = None) -> Problem:
    """17^3 slab: chi = 10^(-4 + 8 k / (n-1)) * (1 + 0.2 (U - 1/2)), eps = 1e-2,
    B = 1, 16 x 16 directions, tolerance 1e-8.

    ``uniform=True`` sets U = 1/2 (horizontally uniform slab)."""
    rng = np.random.default_rng(SEED_BASE + 1 if seed is None else seed)
    nz = ny = nx = n
    k = _depth(nz)
    U = rng.random((nz, ny, nx))
    if uniform:
        U[:] = 0.5
    chi = 10.0 ** (-4.0 + 8.0 * k / (nz - 1)) * (1.0 + 0.2 * (U - 0.5))
    mu, phi, w = quadrature(n_theta, n_phi)
    return Problem(nx, ny, nz, np.ascontiguousarray(chi),
                   np.full((nz, ny, nx), eps), np.ones((nz, ny, nx)),
                   mu, phi, w, tol=1e-8, name=f"slab {n}^3 eps={eps:g}")


def slab_65(n: int = 65, n_theta: int = 32, n_phi: int = 32,
            seed: Optional[int] = None) -> Problem:
    """65^3 slab: chi = 10^(-4 + 8 k / 64) * exp(0.3 N(0,1)) per voxel,
    eps = 10^(-4 U) per voxel, B = (1 + k/64)^4, 32 x 32 directions,
    tolerance 1e-8."""
    rng = np.random.default_rng(SEED_BASE + 2 if seed is None else seed)
    nz = ny = nx = n
    k = _depth(nz)
    Z = float(nz - 1)
    chi = 10.0 ** (-4.0 + 8.0 * k / Z) * np.exp(0.3 * rng.standard_normal((nz, ny, nx)))
    eps = 10.0 ** (-4.0 * rng.random((nz, ny, nx)))
    B = np.broadcast_to((1.0 + k / Z) ** 4, (nz, ny, nx)).copy()
    mu, phi, w = quadrature(n_theta, n_phi)
    return Problem(nx, ny, nz, np.ascontiguousarray(chi), eps, B, mu, phi, w,
                   tol=1e-8, name=f"slab {n}^3 lognormal chi, per-voxel eps")


def slab_precision(n: int = 129, nzz: Optional[int] = None, eps: float = 1e-6,
                   n_theta: int = 64, n_phi: int = 64,
                   seed: Optional[int] = None) -> Problem:
    """Strong-scattering slab: chi = 10^(-4 + 8 k / (nz-1)) * (1 + 0.2 (U - 1/2)),
    eps = 1e-6, B = 1, 64 x 64 directions (129^3 at full size)."""
    rng = np.random.default_rng(SEED_BASE + 3 if seed is None else seed)
    nx = ny = n
    nz = n if nzz is None else nzz
    k = _depth(nz)
    U = rng.random((nz, ny, nx))
    chi = 10.0 ** (-4.0 + 8.0 * k / (nz - 1)) * (1.0 + 0.2 * (U - 0.5))
    mu, phi, w = quadrature(n_theta, n_phi)
    return Problem(nx, ny, nz, np.ascontiguousarray(chi),
                   np.full((nz, ny, nx), eps), np.ones((nz, ny, nx)),
                   mu, phi, w, tol=1e-8, name=f"slab {nx}x{ny}x{nz} eps={eps:g}")


def batch_65(n_lambda: int = 512, n: int = 65, n_theta: int = 32, n_phi: int = 32,
             seed: Optional[int] = None) -> List[Problem]:
    """Wavelength batch: each point uses the 65^3 slab's chi field and B,
    chi scaled by s = 10^(-2 + 4 U) and a constant eps = 10^(-5 + 5 U)."""
    base = slab_65(n=n, n_theta=n_theta, n_phi=n_phi)
    rng = np.random.default_rng(SEED_BASE + 4 if seed is None else seed)
    s = 10.0 ** (-2.0 + 4.0 * rng.random(n_lambda))
    e = 10.0 ** (-5.0 + 5.0 * rng.random(n_lambda))
    out = []
    for lam in range(n_lambda):
        out.append(Problem(base.nx, base.ny, base.nz, base.chi * s[lam],
                           np.full_like(base.chi, e[lam]), base.B, base.mu,
                           base.phi, base.w, tol=1e-8,
                           name=f"lambda {lam}: chi x {s[lam]:.3g}, eps {e[lam]:.3g}"))
    return out


def batch_uneven(sizes=((257, 257, 129, 8), (129, 129, 129, 24), (65, 65, 65, 32)),
                 n_theta: int = 64, n_phi: int = 64, seed: Optional[int] = None,
                 materialise: bool = True) -> List[Problem]:
    """Uneven batch: 8 x 257^2x129, 24 x 129^3, 32 x 65^3 slabs, chi from
    the strong-scattering law scaled by s = 10^(-2 + 4 U), constant
    eps = 10^(-5 + 5 U) per wavelength."""
    rng = np.random.default_rng(SEED_BASE + 5 if seed is None else seed)
    mu, phi, w = quadrature(n_theta, n_phi)
    out = []
    lam = 0
    for (nx, ny, nz, count) in sizes:
        for _ in range(count):
            s = 10.0 ** (-2.0 + 4.0 * rng.random())
            e = 10.0 ** (-5.0 + 5.0 * rng.random())
            sub = np.random.default_rng([SEED_BASE + 5, lam])
            k = _depth(nz)
            if materialise:
                U = sub.random((nz, ny, nx))
                chi = s * 10.0 ** (-4.0 + 8.0 * k / (nz - 1)) * (1.0 + 0.2 * (U - 0.5))
                eps = np.full((nz, ny, nx), e)
                B = np.ones((nz, ny, nx))
            else:
                chi = eps = B = None
            out.append(Problem(nx, ny, nz, chi, eps, B, mu, phi, w, tol=1e-8,
                               name=f"lambda {lam}: {nx}x{ny}x{nz} chi x {s:.3g} eps {e:.3g}"))
            lam += 1
    return out


def random_slab(nx: int, ny: int, nz: int, n_theta: int = 4, n_phi: int = 4,
                seed: int = 7, eps_range=(1e-2, 1.0), chi_decades: float = 3.0,
                top_bc: int = BC_ZERO, bottom_bc: int = BC_PLANCK,
                dx: float = 1.0, dy: float = 1.0, dz: float = 1.0) -> Problem:
    """Small random slab for parity and edge cases: log-uniform chi over
    ``chi_decades`` decades around 1, log-uniform eps, B in [1, 2)."""
    rng = np.random.default_rng(seed)
    chi = 10.0 ** (chi_decades * (rng.random((nz, ny, nx)) - 0.5))
    lo, hi = math.log10(eps_range[0]), math.log10(eps_range[1])
    eps = 10.0 ** (lo + (hi - lo) * rng.random((nz, ny, nx)))
    B = 1.0 + rng.random((nz, ny, nx))
    mu, phi, w = quadrature(n_theta, n_phi)
    return Problem(nx, ny, nz, chi, eps, B, mu, phi, w, dx=dx, dy=dy, dz=dz,
                   top_bc=top_bc, bottom_bc=bottom_bc, tol=1e-10,
                   name=f"random {nx}x{ny}x{nz}")


PRESETS = {
    "slab17": slab_small,
    "slab65": slab_65,
    "slab129_eps1e-6": slab_precision,
}
