"""Oracle for the Cartesian -> radial SHO transform (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import this
module.  It shares no code with the CUDA library.

Sec. 2.4 (eq. SHO-transform-Cartesian-to-radial): within each energy shell nu = nx + ny + nz = 2 nr + l the
Cartesian states Psi_{nx ny nz} (eq. SHO-eigenstate-Cartesian, Sec. 2.2) and the radial states
Psi_{nr l m} = R_{nr l}(r) Y_{l m} (eq. SHO-eigenstate-radial, Sec. 2.3) span the same space, and a unitary
U with Psi_{nx ny nz} = sum_{nr l m} U[nx ny nz][nr l m] Psi_{nr l m} connects them.  For real, orthonormal
bases U[k][j] = <Psi_j^rad | Psi_k^cart>, and projection coefficients transform as
c_rad[j] = sum_k U[k][j] c_cart[k].

Conventions (the paper leaves them open):
  * Y_{l m} real spherical harmonics built from the complex ones with the Condon-Shortley phase:
    m > 0: sqrt(2) (-1)^m Re Y_l^m,  m = 0: Y_l^0,  m < 0: sqrt(2) (-1)^m Im Y_l^{|m|}
    (so m = +1, -1, 0 of l = 1 are the x, y, z orbitals with positive sign);
  * R_{nr l}(r) = N r^l L_nr^{(l + 1/2)}(r^2 / sigma^2) exp(-r^2 / 2 sigma^2) with N > 0 and
    int R^2 r^2 dr = 1 (positive at the origin);
  * radial index order: nu ascending, then l ascending (l = nu mod 2, ..., nu), then m = -l .. l.

U is independent of sigma; it is computed here by Gauss-Hermite quadrature of the products of the two
sets of states (exact for these polynomial-times-Gaussian integrands at n >= numax + 1 nodes per axis),
with the states evaluated from scipy's Laguerre and associated-Legendre functions.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special

from . import basis, nstates


def radial_labels(numax: int):
    """(nr, l, m) of the radial states in the library's order."""
    out = []
    for nu in range(numax + 1):
        for ell in range(nu % 2, nu + 1, 2):
            nr = (nu - ell) // 2
            for m in range(-ell, ell + 1):
                out.append((nr, ell, m))
    return out


def _hermite_fn(n, x):
    """Normalised 1D oscillator function with sigma = 1 (eq. 1HO-eigenstate with its norm)."""
    return special.eval_hermite(n, x) * np.exp(-0.5 * x * x) / math.sqrt(math.sqrt(math.pi) * 2.0 ** n
                                                                       * math.factorial(n))


def _real_ylm(ell, m, theta, phi):
    """Real spherical harmonic Y_{l m}(theta, phi) (convention in the module docstring)."""
    am = abs(m)
    norm = math.sqrt((2 * ell + 1) / (4 * math.pi) * math.factorial(ell - am) / math.factorial(ell + am))
    plm = special.lpmv(am, ell, np.cos(theta))  # includes the Condon-Shortley phase (-1)^m
    if m == 0:
        return norm * plm
    if m > 0:
        return math.sqrt(2.0) * (-1) ** m * norm * plm * np.cos(am * phi)
    return math.sqrt(2.0) * (-1) ** m * norm * plm * np.sin(am * phi)


def _radial_fn(nr, ell, r):
    """R_{nr l}(r) for sigma = 1, normalised so that int R^2 r^2 dr = 1."""
    alpha = ell + 0.5
    # int_0^inf r^(2l+2) L^2 exp(-r^2) dr = Gamma(nr + l + 3/2) / (2 nr!)
    norm = math.sqrt(2.0 * math.factorial(nr) / special.gamma(nr + ell + 1.5))
    return norm * r ** ell * special.eval_genlaguerre(nr, alpha, r * r) * np.exp(-0.5 * r * r)


def radial_value(nr, ell, m, x, y, z, sigma=1.0):
    """Psi_{nr l m} at points (x, y, z) relative to the centre, width sigma (3D L2-normalised)."""
    x, y, z = (np.asarray(v, dtype=np.float64) / sigma for v in (x, y, z))
    r = np.sqrt(x * x + y * y + z * z)
    theta = np.arccos(np.where(r > 0, z / np.where(r > 0, r, 1.0), 1.0))
    phi = np.arctan2(y, x)
    return _radial_fn(nr, ell, r) * _real_ylm(ell, m, theta, phi) / sigma ** 1.5


def radial_matrix(numax: int, nodes: int = None) -> np.ndarray:
    """U[k][j] = <Psi_j^rad | Psi_k^cart> (k in the library's Cartesian order, j in radial_labels order),
    by tensor Gauss-Hermite quadrature with weight exp(-x^2) per axis."""
    n = nodes if nodes is not None else numax + 2
    t, w = special.roots_hermite(n)
    X, Y, Z = np.meshgrid(t, t, t, indexing="ij")
    W = (w[:, None, None] * w[None, :, None] * w[None, None, :]) * np.exp(X * X + Y * Y + Z * Z)
    cart = basis(numax)
    rad = radial_labels(numax)
    N = nstates(numax)
    U = np.zeros((N, N))
    hx = [_hermite_fn(i, t) for i in range(numax + 1)]
    rv = [radial_value(nr, ell, m, X, Y, Z) for (nr, ell, m) in rad]
    for k, (nx, ny, nz) in enumerate(cart):
        ck = hx[nx][:, None, None] * hx[ny][None, :, None] * hx[nz][None, None, :]
        for j in range(N):
            U[k, j] = float(np.sum(W * ck * rv[j]))
    return U


def to_radial(c: np.ndarray, numax: int, inverse: bool = False) -> np.ndarray:
    """c[..., k, b] (Cartesian) -> c[..., j, b] (radial) = sum_k U[k][j] c[k]; inverse maps back (U
    is orthogonal, its inverse is its transpose)."""
    U = radial_matrix(numax)
    c = np.asarray(c, dtype=np.float64)
    return np.einsum("kj,...jb->...kb", U, c) if inverse else np.einsum("kj,...kb->...jb", U, c)
