"""Stored-projector FP64 baseline (the paper's "USU" comparison, Sec. 6) against the oracle (GPU)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, assert_coeff_close, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("periodic", [True, False])
def test_usu_matches_oracle(periodic):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(200)
    grid, h, numax, cube = (36, 40, 32), 0.2, 5, 16
    pos, sig = workloads.random_atoms(rng, 5, tuple(n * h for n in grid), periodic, min_sep=1.0)
    psi = rng.standard_normal((32, 40, 36, 40))
    c = rng.standard_normal((5, oracle.nstates(numax), 40))
    proj = api.usu_build(pos, sig, numax, cube, grid, h, periodic)
    psi_d = torch.from_numpy(psi).cuda()
    got = api.usu_project(psi_d, proj, pos, sig, numax, cube, h, periodic).cpu().numpy()
    ref = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube)
    assert_coeff_close(got, ref, TOL_FP64)
    api.usu_add(psi_d, torch.from_numpy(c).cuda(), proj, pos, sig, numax, cube, h, periodic)
    ref2 = oracle.add(grid, h, periodic, psi, pos, sig, numax, cube, c)
    assert rel_norm(psi_d.cpu().numpy() - psi, ref2 - psi) <= TOL_FP64


def test_usu_rejects_large_numax():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api, ShoError
    with pytest.raises(ShoError):
        api.usu_build(np.zeros((1, 3)), [1.0], 6, 16, (16, 16, 16), 0.25, True)


def test_usu_truncated_projector_set():
    """18 stored projectors (the first 18 states of the numax-4 basis, the size of the s, s*, p, p*, d, d*
    set of Sec. 6): the oracle's numax-4 projection restricted to those states, and its expansion with the
    remaining coefficients zero."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(201)
    grid, h, numax, cube, nproj = (40, 36, 34), 0.2, 4, 16, 18
    pos, sig = workloads.random_atoms(rng, 4, tuple(n * h for n in grid), False, min_sep=1.0)
    psi = rng.standard_normal((34, 36, 40, 33))
    c = rng.standard_normal((4, nproj, 33))
    proj = api.usu_build(pos, sig, numax, cube, grid, h, False, nproj=nproj)
    assert tuple(proj.shape) == (4, cube ** 3, nproj)
    psi_d = torch.from_numpy(psi).cuda()
    got = api.usu_project(psi_d, proj, pos, sig, numax, cube, h, False).cpu().numpy()
    ref = oracle.project(grid, h, False, psi, pos, sig, numax, cube)[:, :nproj]
    assert_coeff_close(got, ref, TOL_FP64)
    cfull = np.zeros((4, oracle.nstates(numax), 33))
    cfull[:, :nproj] = c
    api.usu_add(psi_d, torch.from_numpy(c).cuda(), proj, pos, sig, numax, cube, h, False)
    ref2 = oracle.add(grid, h, False, psi, pos, sig, numax, cube, cfull)
    assert rel_norm(psi_d.cpu().numpy() - psi, ref2 - psi) <= TOL_FP64


def test_usu_rejects_unsupported_nproj():
    require_gpu()
    from paper_1905_00480_gb300 import api, ShoError
    for nproj in (0, 17, 36):
        with pytest.raises(ShoError):
            api.usu_build(np.zeros((1, 3)) + 1.0, [1.0], 4, 16, (16, 16, 16), 0.25, True, nproj=nproj)


@pytest.mark.parametrize("nbands,nproj", [(40, 18), (42, 18), (45, 35), (40, 56)])
def test_usu_float(nbands, nproj):
    """Float stored projectors (the paper's float column of Table 2): projection and expansion against
    the FP64 oracle run on the same FP32-rounded inputs; the 32^3-term sums in FP32 bound the error by
    a few 1e-6 norm-wise.  40 / 42 / 45 bands take 4, 2 and 1 bands per lane."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(202 + nbands)
    grid, h, cube = (36, 40, 32), 0.2, 16
    numax = next(v for v in range(6) if oracle.nstates(v) >= nproj)
    pos, sig = workloads.random_atoms(rng, 5, tuple(n * h for n in grid), True, min_sep=1.0)
    psi = rng.standard_normal((32, 40, 36, nbands)).astype(np.float32)
    c = rng.standard_normal((5, nproj, nbands)).astype(np.float32)
    proj = api.usu_build(pos, sig, numax, cube, grid, h, True, nproj=nproj, dtype=torch.float32)
    psi_d = torch.from_numpy(psi).cuda()
    got = api.usu_project(psi_d, proj, pos, sig, numax, cube, h, True).double().cpu().numpy()
    ref = oracle.project(grid, h, True, psi.astype(np.float64), pos, sig, numax, cube)[:, :nproj]
    assert rel_norm(got, ref) <= 2e-5
    cfull = np.zeros((5, oracle.nstates(numax), nbands))
    cfull[:, :nproj] = c
    api.usu_add(psi_d, torch.from_numpy(c).cuda(), proj, pos, sig, numax, cube, h, True)
    ref2 = oracle.add(grid, h, True, psi.astype(np.float64), pos, sig, numax, cube, cfull)
    assert rel_norm(psi_d.double().cpu().numpy() - psi, ref2 - psi) <= 2e-5


def test_usu_positions_outside_periodic_box():
    """Periodic grid, atoms given several box lengths outside the cell: the stored-projector kernels wrap
    the cube origin and agree with the oracle."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(203)
    grid, h, numax, cube = (36, 40, 32), 0.2, 3, 16
    L = np.array(grid) * h
    pos, sig = workloads.random_atoms(rng, 4, tuple(L), True, min_sep=1.0)
    pos = pos + np.array([[-2, 0, 3], [5, -1, 0], [0, 0, -7], [1, 1, 1]]) * L
    psi = rng.standard_normal((32, 40, 36, 8))
    proj = api.usu_build(pos, sig, numax, cube, grid, h, True)
    got = api.usu_project(torch.from_numpy(psi).cuda(), proj, pos, sig, numax, cube, h, True).cpu().numpy()
    assert_coeff_close(got, oracle.project(grid, h, True, psi, pos, sig, numax, cube), TOL_FP64)
