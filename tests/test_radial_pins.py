"""Pins of the oracle's Cartesian -> radial transform (eq. SHO-transform-Cartesian-to-radial, Sec. 2.4).

Checked against facts fixed by the mathematics rather than against the oracle itself:
  * the shell rule: U[k][j] = 0 unless nx + ny + nz = 2 nr + l (Sec. 2.4);
  * unitarity: both bases are orthonormal, so U^T U = 1 (a wrong norm of R, Y or phi breaks it);
  * closed forms of the lowest shells, derived by hand from the Hermite and Laguerre polynomials:
      nu = 0   Psi_000 = Psi_{0 0 0}
      nu = 1   x, y, z orbitals: Psi_100 = p(m=+1), Psi_010 = p(m=-1), Psi_001 = p(m=0)
      nu = 2   Psi_110 = d(m=-2) (xy), Psi_101 = d(m=+1) (xz), Psi_011 = d(m=-1) (yz);
               H_2 = 4x^2 - 2 gives Psi_200 + Psi_020 + Psi_002 ~ (r^2 - 3/2) e^{-r^2/2}, while
               L_1^{(1/2)}(r^2) = 3/2 - r^2, so <2s | Psi_200> = -1/sqrt(3);
               d(m=0) ~ 2z^2 - x^2 - y^2 = (2 Psi_002 - Psi_200 - Psi_020)/sqrt(6) up to normalisation,
               so <d0 | Psi_002> = 2/sqrt(6), <d0 | Psi_200> = -1/sqrt(6);
               d(m=+2) ~ x^2 - y^2, so <d2 | Psi_200> = 1/sqrt(2), <d2 | Psi_020> = -1/sqrt(2);
  * quadrature exactness: more nodes do not change U;
  * a radial state sampled on a fine grid and projected with the direct-summation oracle gives the unit
    vector of that state after the transform (eq. SHO-basis: both truncated bases span one space).
"""
import math

import numpy as np
import pytest

import oracle
from oracle import radial


def _idx(numax):
    cart = {tuple(int(v) for v in s): k for k, s in enumerate(oracle.basis(numax))}
    rad = {s: j for j, s in enumerate(radial.radial_labels(numax))}
    return cart, rad


def test_shell_sizes_and_labels():
    for numax in range(7):
        labels = radial.radial_labels(numax)
        assert len(labels) == oracle.nstates(numax)
        assert len(set(labels)) == len(labels)
        for nr, ell, m in labels:
            assert 2 * nr + ell <= numax and -ell <= m <= ell


@pytest.mark.parametrize("numax", [0, 1, 2, 3, 4, 5, 6])
def test_unitary_and_shell_block_diagonal(numax):
    U = radial.radial_matrix(numax)
    assert np.max(np.abs(U.T @ U - np.eye(len(U)))) < 1e-12
    cart = oracle.basis(numax)
    rad = radial.radial_labels(numax)
    for k, (nx, ny, nz) in enumerate(cart):
        for j, (nr, ell, m) in enumerate(rad):
            if nx + ny + nz != 2 * nr + ell:
                assert abs(U[k, j]) < 1e-14


def test_lowest_shells_closed_forms():
    U = radial.radial_matrix(2)
    c, r = _idx(2)
    assert U[c[(0, 0, 0)], r[(0, 0, 0)]] == pytest.approx(1.0, abs=1e-14)
    assert U[c[(1, 0, 0)], r[(0, 1, 1)]] == pytest.approx(1.0, abs=1e-14)
    assert U[c[(0, 1, 0)], r[(0, 1, -1)]] == pytest.approx(1.0, abs=1e-14)
    assert U[c[(0, 0, 1)], r[(0, 1, 0)]] == pytest.approx(1.0, abs=1e-14)
    assert U[c[(1, 1, 0)], r[(0, 2, -2)]] == pytest.approx(1.0, abs=1e-14)
    assert U[c[(1, 0, 1)], r[(0, 2, 1)]] == pytest.approx(1.0, abs=1e-14)
    assert U[c[(0, 1, 1)], r[(0, 2, -1)]] == pytest.approx(1.0, abs=1e-14)
    for s in [(2, 0, 0), (0, 2, 0), (0, 0, 2)]:
        assert U[c[s], r[(1, 0, 0)]] == pytest.approx(-1.0 / math.sqrt(3.0), abs=1e-14)
    assert U[c[(0, 0, 2)], r[(0, 2, 0)]] == pytest.approx(2.0 / math.sqrt(6.0), abs=1e-14)
    assert U[c[(2, 0, 0)], r[(0, 2, 0)]] == pytest.approx(-1.0 / math.sqrt(6.0), abs=1e-14)
    assert U[c[(2, 0, 0)], r[(0, 2, 2)]] == pytest.approx(1.0 / math.sqrt(2.0), abs=1e-14)
    assert U[c[(0, 2, 0)], r[(0, 2, 2)]] == pytest.approx(-1.0 / math.sqrt(2.0), abs=1e-14)


def test_quadrature_order_does_not_matter():
    for numax in (3, 5):
        assert np.max(np.abs(radial.radial_matrix(numax) - radial.radial_matrix(numax, nodes=numax + 6))) < 1e-13


def test_sampled_radial_state_projects_to_unit_vector():
    """Wide cube, fine spacing (the discrete-orthonormality regime of the basis pins): a sampled radial
    state Psi_{nr l m} projects (oracle direct summation) and transforms to e_j."""
    numax, sigma, h, C = 3, 0.42, 0.1, 64
    X = np.array([[C * h / 2 + 0.013, C * h / 2 - 0.021, C * h / 2 + 0.007]])
    j = np.arange(C) * h                                                # grid points x_j = j h
    xx, yy, zz = np.meshgrid(j - X[0, 0], j - X[0, 1], j - X[0, 2], indexing="ij")
    labels = radial.radial_labels(numax)
    for js in (0, 4, 11, 15, 19):
        nr, ell, m = labels[js]
        vals = radial.radial_value(nr, ell, m, xx, yy, zz, sigma)       # [x][y][z]
        psi = np.transpose(vals, (2, 1, 0))[..., None]                  # [z][y][x][1]
        c = oracle.project((C, C, C), h, False, psi, X, [sigma], numax, C)
        crad = radial.to_radial(c[0], numax)[:, 0]
        e = np.zeros(len(labels))
        e[js] = 1.0
        assert np.max(np.abs(crad - e)) < 1e-10, (js, labels[js])
