"""FP64 CPU oracle for SHO projection / expansion / forces (test infrastructure only).

Only the test suite, ``__graft_entry__.smoke()`` and the CPU-baseline leg of ``bench.py`` may import
this package.  It shares no code with the CUDA library in ``paper_1905_00480_gb300`` and never calls
it.  The arithmetic lives in ``sho_oracle.c`` (plain C, FP64 with long-double polynomials); this
module only compiles it with gcc and marshals numpy arrays through ctypes.

Definitions follow Baumeister & Tsukamoto (PASC'19): eq. 1HO-eigenstate and eq.
SHO-eigenstate-Cartesian (Sec. 2.2) for the functions, eq. SHO-basis / SHO_basis_size (Sec. 2.5) for
the truncated basis, the three steps of the non-local action (Sec. 3.2) for projection and expansion.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sho_oracle.c")
_OUT_DIR = os.path.join(_HERE, "_build")
_LIB_PATH = os.path.join(_OUT_DIR, "liboracle.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile sho_oracle.c into a shared library with gcc (OpenMP, no FMA contraction)."""
    os.makedirs(_OUT_DIR, exist_ok=True)
    if (not force and os.path.exists(_LIB_PATH)
            and os.path.getmtime(_LIB_PATH) >= os.path.getmtime(_SRC)):
        return _LIB_PATH
    tmp = _LIB_PATH + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-o", tmp, _SRC, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _LIB_PATH)
    return _LIB_PATH


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            i64p = ctypes.POINTER(ctypes.c_int64)
            dp = ctypes.POINTER(ctypes.c_double)
            ip = ctypes.POINTER(ctypes.c_int)
            lib.oracle_set_threads.argtypes = [ctypes.c_int]
            lib.oracle_set_threads.restype = ctypes.c_int
            lib.oracle_nstates.argtypes = [ctypes.c_int]
            lib.oracle_nstates.restype = ctypes.c_int
            lib.oracle_basis.argtypes = [ctypes.c_int, ip]
            lib.oracle_basis.restype = ctypes.c_int
            lib.oracle_hermite.argtypes = [ctypes.c_int, ctypes.c_double]
            lib.oracle_hermite.restype = ctypes.c_double
            lib.oracle_phi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.oracle_phi.restype = ctypes.c_double
            lib.oracle_dphi.argtypes = [ctypes.c_int, ctypes.c_double, ctypes.c_double]
            lib.oracle_dphi.restype = ctypes.c_double
            common = [ip, ctypes.c_double, ctypes.c_int]
            lib.oracle_project.argtypes = common + [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                    ctypes.c_int, dp]
            lib.oracle_add.argtypes = common + [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                ctypes.c_int, dp]
            lib.oracle_forces.argtypes = common + [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                   ctypes.c_int, dp, dp]
            lib.oracle_expand_points.argtypes = common + [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                          ctypes.c_int, dp, ctypes.c_int, i64p, dp]
            lib.oracle_project_bloch.argtypes = [ip, ctypes.c_double, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp,
                                                 ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_add_bloch.argtypes = [ip, ctypes.c_double, dp, dp, ctypes.c_int, ctypes.c_int, dp, dp,
                                             ctypes.c_int, ctypes.c_int, dp]
            lib.oracle_project_r.argtypes = common + [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                      ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_add_r.argtypes = common + [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                  ctypes.c_int, ctypes.c_double, dp]
            lib.oracle_forces_r.argtypes = common + [dp, ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                     ctypes.c_int, ctypes.c_double, dp, dp]
            lib.oracle_expand_points_r.argtypes = common + [ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int,
                                                            ctypes.c_int, ctypes.c_double, dp, ctypes.c_int, i64p,
                                                            dp]
            for f in (lib.oracle_project, lib.oracle_add, lib.oracle_forces, lib.oracle_expand_points,
                      lib.oracle_project_bloch, lib.oracle_add_bloch, lib.oracle_project_r, lib.oracle_add_r,
                      lib.oracle_forces_r, lib.oracle_expand_points_r):
                f.restype = ctypes.c_int
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _grid(n):
    return (ctypes.c_int * 3)(*[int(v) for v in n])


def _f64(a, shape=None):
    a = np.ascontiguousarray(a, dtype=np.float64)
    if shape is not None and a.shape != tuple(shape):
        raise ValueError(f"expected shape {tuple(shape)}, got {a.shape}")
    return a


def _check(rc, what):
    if rc != 0:
        raise ValueError(f"oracle {what} rejected its arguments (code {rc})")


def set_threads(n: int) -> int:
    """Set the oracle's OpenMP thread count (n <= 0 leaves it); returns the count now in effect."""
    return int(_load().oracle_set_threads(int(n)))


def nstates(numax: int) -> int:
    """Size of the truncated basis, eq. SHO_basis_size (Sec. 2.5)."""
    return int(_load().oracle_nstates(int(numax)))


def basis(numax: int) -> np.ndarray:
    """(N, 3) array of (nx, ny, nz), nz outer / ny middle / nx inner, nx+ny+nz <= numax."""
    n = nstates(numax)
    out = np.zeros((n, 3), dtype=np.int32)
    _load().oracle_basis(int(numax), out.ctypes.data_as(ctypes.POINTER(ctypes.c_int)))
    return out


def hermite(n: int, x: float) -> float:
    """Physicists' Hermite polynomial H_n(x) from its explicit power sum."""
    return float(_load().oracle_hermite(int(n), float(x)))


def phi(n: int, u: float, sigma: float) -> float:
    """L2-normalised 1D oscillator function (eq. 1HO-eigenstate with its normalisation)."""
    return float(_load().oracle_phi(int(n), float(u), float(sigma)))


def dphi(n: int, u: float, sigma: float) -> float:
    """d phi_n / du."""
    return float(_load().oracle_dphi(int(n), float(u), float(sigma)))


def project(grid, h, periodic, psi, pos, sigma, numax, cube, rprj=0.0):
    """c[a][k][b] = h^3 sum over the atom's cube of Psi_k(u) psi[j][b]; psi is [Nz][Ny][Nx][B].
    rprj > 0: only cube points with (ux^2 + uy^2) + uz^2 <= rprj^2 (FP64, in that order) contribute."""
    n = [int(v) for v in grid]
    psi = _f64(psi)
    B = psi.shape[-1]
    assert psi.shape == (n[2], n[1], n[0], B), psi.shape
    pos = _f64(pos).reshape(-1, 3)
    sigma = _f64(sigma).reshape(-1)
    A = pos.shape[0]
    N = nstates(numax)
    c = np.zeros((A, N, B), dtype=np.float64)
    rc = _load().oracle_project_r(_grid(n), float(h), int(bool(periodic)), _dp(psi), B, A, _dp(pos), _dp(sigma),
                                  int(numax), int(cube), float(rprj), _dp(c))
    _check(rc, "project")
    return c


def add(grid, h, periodic, psi, pos, sigma, numax, cube, coeff, rprj=0.0):
    """Returns psi + sum_a sum_k c[a][k][b] Psi_k (the input array is not modified); rprj as in project."""
    n = [int(v) for v in grid]
    out = np.array(psi, dtype=np.float64, copy=True, order="C")
    B = out.shape[-1]
    assert out.shape == (n[2], n[1], n[0], B), out.shape
    pos = _f64(pos).reshape(-1, 3)
    sigma = _f64(sigma).reshape(-1)
    A = pos.shape[0]
    coeff = _f64(coeff, (A, nstates(numax), B))
    rc = _load().oracle_add_r(_grid(n), float(h), int(bool(periodic)), _dp(out), B, A, _dp(pos), _dp(sigma),
                              int(numax), int(cube), float(rprj), _dp(coeff))
    _check(rc, "add")
    return out


def expand_points(grid, h, periodic, pos, sigma, numax, cube, coeff, points, rprj=0.0):
    """Expansion evaluated at selected flat grid indices: returns [P][B]; rprj as in project."""
    n = [int(v) for v in grid]
    pos = _f64(pos).reshape(-1, 3)
    sigma = _f64(sigma).reshape(-1)
    A = pos.shape[0]
    coeff = _f64(coeff)
    B = coeff.shape[-1]
    assert coeff.shape == (A, nstates(numax), B)
    pts = np.ascontiguousarray(points, dtype=np.int64)
    out = np.zeros((pts.size, B), dtype=np.float64)
    rc = _load().oracle_expand_points_r(_grid(n), float(h), int(bool(periodic)), B, A, _dp(pos), _dp(sigma),
                                        int(numax), int(cube), float(rprj), _dp(coeff), int(pts.size),
                                        pts.ctypes.data_as(ctypes.POINTER(ctypes.c_int64)), _dp(out))
    _check(rc, "expand_points")
    return out


def forces(grid, h, periodic, psi, pos, sigma, numax, cube, dEdc, rprj=0.0):
    """dE/dX[a][d] = sum_b sum_k dEdc[a][k][b] dc[a][k][b]/dX_{a,d} (cube origin held fixed; with rprj > 0
    the set of points inside the sphere is held fixed as well)."""
    n = [int(v) for v in grid]
    psi = _f64(psi)
    B = psi.shape[-1]
    pos = _f64(pos).reshape(-1, 3)
    sigma = _f64(sigma).reshape(-1)
    A = pos.shape[0]
    dEdc = _f64(dEdc, (A, nstates(numax), B))
    out = np.zeros((A, 3), dtype=np.float64)
    rc = _load().oracle_forces_r(_grid(n), float(h), int(bool(periodic)), _dp(psi), B, A, _dp(pos), _dp(sigma),
                                 int(numax), int(cube), float(rprj), _dp(dEdc), _dp(out))
    _check(rc, "forces")
    return out


def project_bloch(grid, h, kvec, psi, pos, sigma, numax, cube):
    """Bloch projection on a periodic grid: psi complex [Nz][Ny][Nx][B]; returns complex [A][N][B] with
    c = h^3 sum_i Psi_k(u_i) e^{+i k.T_i} psi[j(i)], T_i the lattice translation of cube point i."""
    n = [int(v) for v in grid]
    psi = np.ascontiguousarray(psi, dtype=np.complex128)
    B = psi.shape[-1]
    assert psi.shape == (n[2], n[1], n[0], B), psi.shape
    pos = _f64(pos).reshape(-1, 3)
    sigma = _f64(sigma).reshape(-1)
    A = pos.shape[0]
    N = nstates(numax)
    c = np.zeros((A, N, B), dtype=np.complex128)
    k = _f64(kvec).reshape(3)
    rc = _load().oracle_project_bloch(_grid(n), float(h), _dp(k), _dp(psi.view(np.float64)), B, A, _dp(pos),
                                      _dp(sigma), int(numax), int(cube), _dp(c.view(np.float64)))
    _check(rc, "project_bloch")
    return c


def add_bloch(grid, h, kvec, psi, pos, sigma, numax, cube, coeff):
    """Returns psi + sum_a sum_k c Psi_k e^{-i k.T} (complex; the input is not modified)."""
    n = [int(v) for v in grid]
    out = np.array(psi, dtype=np.complex128, copy=True, order="C")
    B = out.shape[-1]
    pos = _f64(pos).reshape(-1, 3)
    sigma = _f64(sigma).reshape(-1)
    A = pos.shape[0]
    coeff = np.ascontiguousarray(coeff, dtype=np.complex128)
    assert coeff.shape == (A, nstates(numax), B)
    k = _f64(kvec).reshape(3)
    rc = _load().oracle_add_bloch(_grid(n), float(h), _dp(k), _dp(out.view(np.float64)), B, A, _dp(pos),
                                  _dp(sigma), int(numax), int(cube), _dp(coeff.view(np.float64)))
    _check(rc, "add_bloch")
    return out
