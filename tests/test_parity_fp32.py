"""FP32 CUDA-core form (FP32 and BF16 storage) against the FP64 oracle run on the same storage-rounded
inputs (GPU).  Tolerances are stated in tests/helpers.py (TOL_FP32)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, assert_coeff_close, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _case(grid, h, periodic, natoms, numax, nbands, seed):
    rng = np.random.default_rng(seed)
    box = tuple(n * h for n in grid)
    pos, sig = workloads.random_atoms(rng, natoms, box, periodic, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return pos, sig, psi, c


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("periodic", [True, False])
def test_fp32_form(storage, periodic):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    grid, h, numax, cube = (48, 40, 44), 0.2, 5, 32
    pos, sig, psi, c = _case(grid, h, periodic, 6, numax, 72, seed=101)
    psi_d = torch.from_numpy(psi).cuda().to(tdt)
    psi_r = psi_d.double().cpu().numpy()          # storage-rounded input seen by the kernel
    c_d = torch.from_numpy(c).cuda().float()
    c_r = c_d.double().cpu().numpy()
    got = api.project(psi_d, pos, sig, numax, cube, h, periodic, prec="fp32").double().cpu().numpy()
    ref = oracle.project(grid, h, periodic, psi_r, pos, sig, numax, cube)
    assert_coeff_close(got, ref, TOL_FP32)
    if storage == "f32":
        out = psi_d.clone()
        api.add(out, c_d, pos, sig, numax, cube, h, periodic, prec="fp32")
        ref2 = oracle.add(grid, h, periodic, psi_r, pos, sig, numax, cube, c_r)
        assert rel_norm(out.double().cpu().numpy() - psi_r, ref2 - psi_r) <= TOL_FP32
    f = api.forces(psi_d, c_d, pos, sig, numax, cube, h, periodic, prec="fp32").cpu().numpy()
    ref3 = oracle.forces(grid, h, periodic, psi_r, pos, sig, numax, cube, c_r)
    assert rel_max(f, ref3) <= 10 * TOL_FP32


def test_bf16_storage_expansion_rounding():
    """BF16 psi: the expansion result is accumulated in FP32 and rounded once to BF16 on store: per element
    at most 2^-9 |result| from the rounding (2^-8 allowed) plus the FP32 accumulation error."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, numax, cube = (40, 40, 40), 0.2, 3, 16
    pos, sig, psi, c = _case(grid, h, True, 5, numax, 32, seed=102)
    psi_d = torch.from_numpy(psi).cuda().to(torch.bfloat16)
    psi_r = psi_d.double().cpu().numpy()
    c_d = torch.from_numpy(c).cuda().float()
    out = psi_d.clone()
    api.add(out, c_d, pos, sig, numax, cube, h, True, prec="fp32")
    ref = oracle.add(grid, h, True, psi_r, pos, sig, numax, cube, c_d.double().cpu().numpy())
    err = np.abs(out.double().cpu().numpy() - ref)
    assert np.all(err <= 2.0 ** -8 * np.abs(ref) + TOL_FP32 * np.abs(ref).max())


@pytest.mark.parametrize("storage,nbands", [("f32", 40), ("bf16", 56), ("f32", 4)])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "3xtf32", "bf16", "split_fp16"])
@pytest.mark.parametrize("periodic", [True, False])
def test_streaming_kernels_ragged_tiles(storage, nbands, prec, periodic):
    """Band counts with 16-byte rows take the cp.async row pipeline (projection) and the block gather
    (expansion); 40 / 56 bands leave a partial last 32-band tile, 4 bands a single partial tile."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    from test_parity_tc import TOL
    tol = TOL_FP32 if prec == "fp32" else TOL[prec]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[storage]
    grid, h, numax, cube = (44, 40, 36), 0.2, 5, 32
    pos, sig, psi, c = _case(grid, h, periodic, 5, numax, nbands, seed=400 + nbands)
    psi_d = torch.from_numpy(psi).cuda().to(tdt)
    psi_r = psi_d.double().cpu().numpy()
    got = api.project(psi_d, pos, sig, numax, cube, h, periodic, prec=prec).double().cpu().numpy()
    ref = oracle.project(grid, h, periodic, psi_r, pos, sig, numax, cube)
    assert rel_norm(got, ref) <= tol
    c_d = torch.from_numpy(c).cuda().float()
    out = torch.zeros(psi.shape, dtype=torch.float32, device="cuda")
    api.add(out, c_d, pos, sig, numax, cube, h, periodic, prec=prec)
    ref2 = oracle.add(grid, h, periodic, np.zeros_like(psi), pos, sig, numax, cube, c_d.double().cpu().numpy())
    assert rel_norm(out.double().cpu().numpy(), ref2) <= tol


@pytest.mark.parametrize("numax", [8, 9])
def test_streaming_fp32_high_numax(numax):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, cube = (40, 40, 40), 0.2, 32
    pos, sig, psi, c = _case(grid, h, True, 3, numax, 32, seed=500 + numax)
    psi_d = torch.from_numpy(psi).cuda().float()
    got = api.project(psi_d, pos, sig, numax, cube, h, True, prec="fp32").double().cpu().numpy()
    ref = oracle.project(grid, h, True, psi_d.double().cpu().numpy(), pos, sig, numax, cube)
    assert_coeff_close(got, ref, TOL_FP32)
    c_d = torch.from_numpy(c).cuda().float()
    out = psi_d.clone()
    api.add(out, c_d, pos, sig, numax, cube, h, True, prec="fp32")
    ref2 = oracle.add(grid, h, True, psi_d.double().cpu().numpy(), pos, sig, numax, cube, c_d.double().cpu().numpy())
    assert rel_norm(out.double().cpu().numpy() - psi_d.double().cpu().numpy(), ref2 - psi_d.double().cpu().numpy()) <= TOL_FP32
