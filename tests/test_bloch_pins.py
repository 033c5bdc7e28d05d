"""Pins of the oracle's Bloch (complex) projection and expansion on a periodic grid.

The SHO basis spans functions R^3 -> C (Sec. 2.5); for a Bloch wave psi(r + T) = e^{i k.T} psi(r) the
value at a cube point outside the cell is the stored value times the Bloch phase.  Checked against:
  * k = 0: the real oracle applied to the real and imaginary parts;
  * k with k_d L_d a multiple of 2 pi: every lattice phase is 1, so again the k = 0 result;
  * a plane wave e^{i q.r} sampled on the periodic cell with k = q projects exactly as the same plane wave
    sampled, unwrapped, on an open grid three cells wide (the phase logic against plain geometry);
  * the adjoint identity <P psi, c> = h^3 <psi, E c> in the complex inner product.
"""
import numpy as np
import pytest

import oracle
import workloads


def _case(seed, grid=(24, 20, 22), h=0.25, natoms=3, numax=3, nbands=3):
    rng = np.random.default_rng(seed)
    L = np.array(grid) * h
    pos, sig = workloads.random_atoms(rng, natoms, tuple(L), True, min_sep=1.0)
    pos[0] = [0.3 * h + 0.01, L[1] - 0.4 * h, 0.6 * h]     # a cube that wraps on every axis
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)) + 1j * rng.standard_normal(
        (grid[2], grid[1], grid[0], nbands))
    return rng, grid, h, L, pos, sig, numax, psi


def test_zero_k_is_the_real_transform():
    rng, grid, h, L, pos, sig, numax, psi = _case(900)
    cube = 16
    c = oracle.project_bloch(grid, h, [0, 0, 0], psi, pos, sig, numax, cube)
    ref = oracle.project(grid, h, True, psi.real, pos, sig, numax, cube) + 1j * oracle.project(
        grid, h, True, psi.imag, pos, sig, numax, cube)
    assert np.max(np.abs(c - ref)) <= 1e-14 * np.max(np.abs(ref))
    coef = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    out = oracle.add_bloch(grid, h, [0, 0, 0], psi, pos, sig, numax, cube, coef)
    ref2 = oracle.add(grid, h, True, psi.real, pos, sig, numax, cube, coef.real) + 1j * oracle.add(
        grid, h, True, psi.imag, pos, sig, numax, cube, coef.imag)
    assert np.max(np.abs(out - ref2)) <= 1e-14 * np.max(np.abs(ref2))


def test_reciprocal_lattice_k_is_zero_k():
    rng, grid, h, L, pos, sig, numax, psi = _case(901)
    cube = 16
    G = 2 * np.pi * np.array([1, -2, 3]) / L
    c0 = oracle.project_bloch(grid, h, [0, 0, 0], psi, pos, sig, numax, cube)
    cG = oracle.project_bloch(grid, h, G, psi, pos, sig, numax, cube)
    assert np.max(np.abs(cG - c0)) <= 1e-12 * np.max(np.abs(c0))


def test_plane_wave_matches_unwrapped_open_grid():
    rng, grid, h, L, pos, sig, numax, _ = _case(902)
    cube = 16
    q = np.array([0.7, -1.3, 0.4])
    n = np.array(grid)
    x = [np.arange(n[d]) * h for d in range(3)]
    psi = np.exp(1j * (q[2] * x[2][:, None, None] + q[1] * x[1][None, :, None] + q[0] * x[0][None, None, :]))
    c = oracle.project_bloch(grid, h, q, psi[..., None], pos, sig, numax, cube)
    # the same wave on an open grid three cells wide, the cell in the middle
    ext = tuple(int(3 * v) for v in n)
    xe = [np.arange(ext[d]) * h - L[d] for d in range(3)]
    pe = np.exp(1j * (q[2] * xe[2][:, None, None] + q[1] * xe[1][None, :, None] + q[0] * xe[0][None, None, :]))
    pos_e = pos + L
    ref = oracle.project(ext, h, False, pe.real[..., None], pos_e, sig, numax, cube) + 1j * oracle.project(
        ext, h, False, pe.imag[..., None], pos_e, sig, numax, cube)
    assert np.max(np.abs(c - ref)) <= 1e-12 * np.max(np.abs(ref))


def test_adjoint_identity():
    rng, grid, h, L, pos, sig, numax, psi = _case(903)
    cube = 16
    k = np.array([0.9, 0.35, -1.7])
    c = oracle.project_bloch(grid, h, k, psi, pos, sig, numax, cube)
    coef = rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)
    ec = oracle.add_bloch(grid, h, k, np.zeros_like(psi), pos, sig, numax, cube, coef)
    lhs = np.vdot(c, coef)
    rhs = h ** 3 * np.vdot(psi, ec)
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
