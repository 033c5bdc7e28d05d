"""Host logic of the plane sweep (CPU): the row-segment plan of many seeded geometries is checked against
its definition by the library's own checker, and its sweep counts against simple bounds."""
import ctypes

import numpy as np
import pytest

import workloads


def _check(grid, h, periodic, pos, sig, cube):
    from paper_1905_00480_gb300 import _native as N
    g = N.sho_grid()
    g.n[0], g.n[1], g.n[2] = grid
    g.h, g.periodic = h, 1 if periodic else 0
    pos = np.ascontiguousarray(pos, dtype=np.float64).reshape(-1, 3)
    sig = np.ascontiguousarray(sig, dtype=np.float64)
    ni, ns = ctypes.c_int(), ctypes.c_int()
    st = N.lib().sho_plane_plan_check(ctypes.byref(g), len(pos), pos.ctypes.data_as(N._DP), sig.ctypes.data_as(N._DP),
                                      cube, ctypes.byref(ni), ctypes.byref(ns))
    return st, ni.value, ns.value


@pytest.mark.parametrize("seed", range(8))
@pytest.mark.parametrize("periodic", [True, False])
def test_random_geometries(seed, periodic):
    rng = np.random.default_rng(1200 + seed)
    nx, ny, nz = (int(v) for v in rng.integers(34, 72, size=3))
    cube = 32 if min(nx, ny, nz) >= 32 else 16
    h = 0.2
    natoms = int(rng.integers(1, 90))
    box = np.array([nx, ny, nz]) * h
    pos = rng.uniform(-0.2, 1.2, size=(natoms, 3)) * box if not periodic else rng.uniform(0, 1, size=(natoms, 3)) * box
    sig = rng.uniform(0.5, 1.0, size=natoms)
    st, nitems, nsegs = _check((nx, ny, nz), h, periodic, pos, sig, cube)
    assert st == 0
    assert nitems >= (nz if periodic and natoms else 0) or not periodic
    assert nsegs <= 2 * natoms * cube


def test_paper_workloads_single_sweep_mostly():
    """The 160^3 / 512-atom workload needs a second sweep on only a few planes; 96^3 and 128^3 on none."""
    for name, most in (("c160", 170), ("c96", 96), ("c128", 128)):
        w = workloads.WORKLOADS[name]
        pos, sig = workloads.atoms(w)
        st, nitems, _ = _check(w.grid, w.h, w.periodic, pos, sig, w.cube)
        assert st == 0
        assert w.grid[2] <= nitems <= most, (name, nitems)


def test_dense_and_small_grids():
    rng = np.random.default_rng(1300)
    # more overlapping cubes per row than slots: several sweeps per plane
    pos, sig = workloads.random_atoms(rng, 150, (9.6, 9.6, 9.6), True, min_sep=0.5)
    st, nitems, _ = _check((48, 48, 48), 0.2, True, pos, sig, 32)
    assert st == 0 and nitems > 48
    # grid barely longer than the cube: wrapped halves share a warp
    pos, sig = workloads.random_atoms(rng, 20, (7.2, 6.8, 8.0), True, min_sep=0.8)
    st, _, _ = _check((36, 34, 40), 0.2, True, pos, sig, 32)
    assert st == 0
    # grid equal to the cube
    pos, sig = workloads.random_atoms(rng, 6, (6.4, 6.4, 6.4), True, min_sep=1.0)
    st, _, _ = _check((32, 32, 32), 0.2, True, pos, sig, 32)
    assert st == 0
