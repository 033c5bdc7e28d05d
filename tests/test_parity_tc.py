"""Tensor-core precision forms (x-pass on MMA tiles, FP32 accumulation) against the FP64 oracle run on
the same storage-rounded inputs (GPU).

Norm-wise error bounds, from the operand rounding of each form (u = unit roundoff of the operand
type; products of two rounded operands carry ~2u, the 32-term x-pass sums and the FP32 y/z passes add
little on top):
  TF32        u = 2^-11: expected ~5e-4, bound 2e-3
  3XTF32      hi + lo carry 22 bits, lo*lo dropped: expected ~1e-6, bound 1e-5
  BF16        u = 2^-8: expected ~4e-3, bound 1.5e-2
  SPLIT_FP16  hi + scaled lo carry 22 bits: expected ~1e-6, bound 1e-5
Forces difference neighbouring coefficients (ladder relation), which can cancel; their bound is 10x.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu

TOL = {"tf32": 2e-3, "3xtf32": 1e-5, "bf16": 1.5e-2, "split_fp16": 1e-5}


def _case(grid, h, natoms, numax, nbands, seed):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * h for n in grid), True, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return pos, sig, psi, c


@pytest.mark.parametrize("mode", ["tf32", "3xtf32", "bf16", "split_fp16"])
@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_tc_project_add(mode, storage):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    grid, h, numax, cube = (40, 44, 36), 0.2, 7, 32
    pos, sig, psi, c = _case(grid, h, 5, numax, 48, seed=300)
    psi_d = torch.from_numpy(psi).cuda().to(tdt)
    psi_r = psi_d.double().cpu().numpy()
    got = api.project(psi_d, pos, sig, numax, cube, h, True, prec=mode).double().cpu().numpy()
    ref = oracle.project(grid, h, True, psi_r, pos, sig, numax, cube)
    for a in range(len(pos)):
        assert rel_norm(got[a], ref[a]) <= TOL[mode], (a, rel_norm(got[a], ref[a]))
    # expansion into an FP32 buffer (the BF16-stored result is checked for the CUDA-core form)
    c_d = torch.from_numpy(c).cuda().float()
    out = torch.zeros(psi.shape, dtype=torch.float32, device="cuda")
    api.add(out, c_d, pos, sig, numax, cube, h, True, prec=mode)
    ref2 = oracle.add(grid, h, True, np.zeros_like(psi), pos, sig, numax, cube, c_d.double().cpu().numpy())
    assert rel_norm(out.double().cpu().numpy(), ref2) <= TOL[mode]


@pytest.mark.parametrize("mode", ["tf32", "3xtf32", "bf16", "split_fp16"])
def test_tc_ragged_and_clipped(mode):
    """Ragged band tile (37 bands), non-periodic clipped cubes, cube 16, numax 3."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(301)
    grid, h, numax, cube = (24, 20, 28), 0.25, 3, 16
    pos = np.array([[0.3, 0.4, 6.7], [5.5, 2.4, 3.1], [2.0, 4.9, 0.1]])
    sig = np.array([0.7, 0.8, 0.6])
    psi = rng.standard_normal((28, 20, 24, 37))
    c = rng.standard_normal((3, oracle.nstates(numax), 37))
    psi_d = torch.from_numpy(psi).cuda().float()
    got = api.project(psi_d, pos, sig, numax, cube, h, False, prec=mode).double().cpu().numpy()
    ref = oracle.project(grid, h, False, psi_d.double().cpu().numpy(), pos, sig, numax, cube)
    assert rel_norm(got, ref) <= TOL[mode]
    out = torch.zeros_like(psi_d)
    c_d = torch.from_numpy(c).cuda().float()
    api.add(out, c_d, pos, sig, numax, cube, h, False, prec=mode)
    ref2 = oracle.add(grid, h, False, np.zeros_like(psi), pos, sig, numax, cube, c_d.double().cpu().numpy())
    assert rel_norm(out.double().cpu().numpy(), ref2) <= TOL[mode]


@pytest.mark.parametrize("mode", ["tf32", "3xtf32", "bf16", "split_fp16"])
@pytest.mark.parametrize("grid,periodic,numax,cube", [
    ((40, 36, 44), False, 2, 16),    # cubes sticking out of an open box on both sides of x
    ((64, 52, 56), False, 7, 48),    # cube wider than the 32-point tile
    ((34, 40, 36), True, 5, 32),     # periodic grid barely wider than the cube: wrapped tiles
])
def test_tc_block_expansion_edges(mode, grid, periodic, numax, cube):
    """Expansion through the block-gather kernel (band count a multiple of 4) with the x-pass B
    fragments precomputed per atom: tiles where the cube starts before or ends inside the tile, cubes
    wider than a tile, and tiles that see a wrapped cube on both ends."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(310 + cube + numax)
    h = 0.2
    L = np.array(grid) * h
    pos = rng.uniform(0.0, 1.0, size=(5, 3)) * L
    pos[0] = [0.1 * h, 0.5 * L[1], 0.5 * L[2]]          # cube starts before x = 0
    pos[1] = [L[0] - 0.3 * h, 0.3 * L[1], 0.6 * L[2]]   # cube ends past x = Nx
    sig = rng.uniform(0.5, 0.9, size=5)
    nb = 32
    c = rng.standard_normal((5, oracle.nstates(numax), nb))
    out = torch.zeros((grid[2], grid[1], grid[0], nb), dtype=torch.float32, device="cuda")
    c_d = torch.from_numpy(c).cuda().float()
    api.add(out, c_d, pos, sig, numax, cube, h, periodic, prec=mode)
    ref = oracle.add(grid, h, periodic, np.zeros(out.shape), pos, sig, numax, cube, c_d.double().cpu().numpy())
    assert rel_norm(out.double().cpu().numpy(), ref) <= TOL[mode]


@pytest.mark.parametrize("mode", ["tf32", "3xtf32", "bf16", "split_fp16"])
def test_tc_forces(mode):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, numax, cube = (36, 36, 36), 0.2, 5, 32
    pos, sig, psi, c = _case(grid, h, 4, numax, 24, seed=302)
    psi_d = torch.from_numpy(psi).cuda().float()
    c_d = torch.from_numpy(c).cuda().float()
    f = api.forces(psi_d, c_d, pos, sig, numax, cube, h, True, prec=mode).cpu().numpy()
    ref = oracle.forces(grid, h, True, psi_d.double().cpu().numpy(), pos, sig, numax, cube,
                        c_d.double().cpu().numpy())
    assert rel_max(f, ref) <= 10 * TOL[mode]


def test_tc_limits_are_rejected():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api, ShoError
    psi = torch.zeros((32, 32, 32, 8), dtype=torch.float32, device="cuda")
    with pytest.raises(ShoError, match="NUMAX"):
        api.project(psi, np.array([[3.0, 3.0, 3.0]]), [0.7], 8, 16, 0.2, True, prec="tf32")
    with pytest.raises(ShoError, match="CUBE"):
        api.project(psi, np.array([[3.0, 3.0, 3.0]]), [0.7], 3, 24, 0.2, True, prec="bf16")
