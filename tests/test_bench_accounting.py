"""The bench's work accounting (CPU): the distinct covered grid points that every GB/s figure divides
by, counted independently with a set of cube points; the separable flop count per (atom, band) of the
three passes against its closed form for the sizes the measurements quote; the kernel launches per step
of the FP64 forms."""
import os
import sys

import numpy as np
import pytest

import workloads

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _set_count(w, pos):
    """Covered grid points as a set of (z, y, x), cube origin floor(X/h) - C/2 + 1 per axis."""
    pts = set()
    nx, ny, nz = w.grid
    for X in pos:
        o = [int(np.floor(X[d] / w.h)) - w.cube // 2 + 1 for d in range(3)]
        for iz in range(w.cube):
            for iy in range(w.cube):
                for ix in range(w.cube):
                    j = [o[0] + ix, o[1] + iy, o[2] + iz]
                    if w.periodic:
                        j = [j[0] % nx, j[1] % ny, j[2] % nz]
                    elif not (0 <= j[0] < nx and 0 <= j[1] < ny and 0 <= j[2] < nz):
                        continue
                    pts.add((j[2], j[1], j[0]))
    return len(pts)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("seed", [0, 1])
def test_union_points_match_a_set_count(periodic, seed):
    rng = np.random.default_rng(4100 + seed)
    grid = (20, 18, 22)
    w = workloads.Workload(name="t", grid=grid, h=0.25, periodic=periodic, natoms=5, numax=3, cube=8, nbands=4,
                           dtype="f64", seed=seed)
    L = np.array(grid) * w.h
    pos = rng.uniform(-0.1, 1.1, size=(5, 3)) * L if not periodic else rng.uniform(0, 1, size=(5, 3)) * L
    pos[0] = [0.01, L[1] - 0.02, 0.5 * L[2]]   # a cube across the box edge
    assert bench.union_cube_points(w, pos) == _set_count(w, pos)


def test_union_points_single_and_repeated_atom():
    w = workloads.Workload(name="t", grid=(24, 24, 24), h=0.2, periodic=True, natoms=1, numax=3, cube=16, nbands=4,
                           dtype="f64", seed=0)
    X = np.array([[2.31, 1.07, 4.55]])
    assert bench.union_cube_points(w, X) == 16 ** 3
    assert bench.union_cube_points(w, np.vstack([X, X])) == 16 ** 3


@pytest.mark.parametrize("cube,numax,flops", [(32, 3, 283904), (32, 5, 439808), (32, 7, 605696), (32, 9, 782080),
                                              (16, 3, 38528)])
def test_separable_flops_per_atom_band(cube, numax, flops):
    """2 [C^3 (nu+1) + C^2 P + C N] with P = (nu+1)(nu+2)/2 pairs and N states (x-, y-, z-pass FMAs)."""
    nst = (numax + 1) * (numax + 2) * (numax + 3) // 6
    w = workloads.Workload(name="t", grid=(cube, cube, cube), h=0.2, periodic=True, natoms=1, numax=numax, cube=cube,
                           nbands=1, dtype="f64", seed=0)
    alg = bench.algorithmic(w, np.array([[0.1, 0.1, 0.1]]), nst)
    assert alg["flops_prj"] == flops and alg["flops_add"] == flops
    assert alg["union_points"] == cube ** 3
    assert alg["bytes_add"] - alg["bytes_prj"] == cube ** 3 * 8


def test_launches_per_step_of_the_fp64_forms():
    w = workloads.WORKLOADS["c96"]
    assert bench.launches_per_step(None, None, w, "ff64") == 5   # float-float projection, tensor-core expansion
    assert bench.launches_per_step(None, None, w, "ff64", "mma_sync", "mma_sync") == 4  # float-float kernels
    assert bench.launches_per_step(None, None, w, "ff64", "tcgen05", "tcgen05") == 6    # tensor-core x-passes
    assert bench.launches_per_step(None, None, w, "fp64") == 3
