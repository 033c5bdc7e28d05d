"""FP64-accurate projection with the x-pass on the tensor cores by exact digit slicing (GPU).

The tensor-core FF64 projection engine (sho_set_project_kernel tcgen05) against the oracle at the FP64
tolerance on periodic and open grids, numax 0..7, cubes of 16, 24 and 32 points (one and two half
rows, a partial second half) and partial band tiles; against the float-float kernel (close, not bitwise:
the tensor-core path ran); the default engine is the float-float kernel; bit for bit the same from run to run;
and on psi spanning sixteen orders of magnitude (the per-half-row frames)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, assert_coeff_close, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _project(engine, grid, h, periodic, psi, pos, sig, numax, cube):
    from paper_1905_00480_gb300 import api
    hd = api.Handle(0)
    hd.set_project_kernel(engine)
    c = api.project(_t(psi), pos, sig, numax, cube, h, periodic, prec="ff64", handle=hd)
    hd.sync()
    out = c.cpu().numpy()
    hd.close()
    return out


@pytest.mark.parametrize("grid,periodic,numax,cube,nbands,natoms", [
    ((56, 40, 36), True, 5, 32, 64, 6),     # one partial band tile (64 of 128)
    ((44, 38, 30), False, 3, 16, 130, 5),   # clipped cubes; band tiles of 128 + 2; one half row
    ((48, 40, 40), True, 7, 24, 32, 4),     # numax 7 (8 states); a partial second half row
    ((40, 40, 40), True, 0, 16, 8, 6),      # numax 0
    ((48, 34, 32), True, 4, 32, 16, 20),    # many atoms, several per CTA
])
def test_ozaki_projection_matches_oracle(grid, periodic, numax, cube, nbands, natoms):
    require_gpu()
    rng = np.random.default_rng(7500 + 10 * numax + natoms)
    h = 0.2
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * h for n in grid), periodic,
                                      min_sep=0.3 if natoms > 10 else 1.0)
    if not periodic:
        pos[0] = [0.1 * h, 0.5 * grid[1] * h, 0.5 * grid[2] * h]
        pos[1] = [(grid[0] - 0.3) * h, 0.3 * grid[1] * h, (grid[2] - 0.6) * h]
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    got = _project("tcgen05", grid, h, periodic, psi, pos, sig, numax, cube)
    ref = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube)
    assert_coeff_close(got, ref, TOL_FP64)
    ff = _project("mma_sync", grid, h, periodic, psi, pos, sig, numax, cube)
    assert rel_norm(got, ff) <= TOL_FP64
    assert not np.array_equal(got, ff)  # the two engines round differently: the tensor-core path ran
    assert np.array_equal(ff, _project("auto", grid, h, periodic, psi, pos, sig, numax, cube))


def test_ozaki_projection_wide_dynamic_range_and_determinism():
    require_gpu()
    rng = np.random.default_rng(7600)
    grid, h, periodic, numax, cube, nbands = (48, 40, 36), 0.2, True, 5, 32, 32
    pos, sig = workloads.random_atoms(rng, 5, tuple(n * h for n in grid), periodic, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)) * 10.0 ** rng.uniform(-8, 8, (grid[2], grid[1], grid[0], 1))
    runs = [_project("tcgen05", grid, h, periodic, psi, pos, sig, numax, cube) for _ in range(2)]
    assert np.array_equal(runs[0], runs[1])
    ref = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube)
    assert_coeff_close(runs[0], ref, TOL_FP64)
