"""Spherical projector support (the projection spheres of Sec. 6) on the GPU against the oracle's
sphere variant: FP64 and FP64-accurate projection, expansion, forces and non-local action, periodic and
clipped, with spheres that cut through the cube; the stored-projector baseline with the same support;
the forms without sphere support refuse it (GPU)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, assert_coeff_close, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _case(seed, grid=(40, 36, 44), h=0.2, natoms=5, numax=5, nbands=37, periodic=True):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * h for n in grid), periodic, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return grid, h, pos, sig, psi, c


@pytest.mark.parametrize("prec", ["fp64", "ff64"])
@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("R", [1.4, 2.9, 5.0])
def test_sphere_project_add_forces(prec, periodic, R):
    """R = 1.4 and 2.9 cut through the 32-point cube (half-width 3.1-3.3 Bohr at h = 0.2); R = 5.0 holds
    the whole cube (corners at 5.5 Bohr are outside: the sphere still trims them)."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, c = _case(1500, periodic=periodic)
    hd = api.Handle(0)
    hd.set_support_radius(R)
    numax, cube = 5, 32
    got = api.project(torch.from_numpy(psi).cuda(), pos, sig, numax, cube, h, periodic, prec=prec, handle=hd)
    ref = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube, rprj=R)
    assert_coeff_close(got.cpu().numpy(), ref, TOL_FP64)
    out = torch.from_numpy(psi).cuda()
    api.add(out, torch.from_numpy(c).cuda(), pos, sig, numax, cube, h, periodic, prec=prec, handle=hd)
    ref2 = oracle.add(grid, h, periodic, psi, pos, sig, numax, cube, c, rprj=R)
    assert rel_norm(out.cpu().numpy() - psi, ref2 - psi) <= TOL_FP64
    f = api.forces(torch.from_numpy(psi).cuda(), torch.from_numpy(c).cuda(), pos, sig, numax, cube, h, periodic,
                   prec=prec, handle=hd).cpu().numpy()
    ref3 = oracle.forces(grid, h, periodic, psi, pos, sig, numax, cube, c, rprj=R)
    assert rel_max(f, ref3) <= TOL_FP64
    hd.set_support_radius(0.0)   # back to the whole cube
    got0 = api.project(torch.from_numpy(psi).cuda(), pos, sig, numax, cube, h, periodic, prec=prec, handle=hd)
    assert_coeff_close(got0.cpu().numpy(), oracle.project(grid, h, periodic, psi, pos, sig, numax, cube), TOL_FP64)
    hd.close()


def test_sphere_cube64_and_numax9():
    """A 64-point cube (two 32-point halves of each row mask) and the largest basis."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, c = _case(1501, grid=(72, 68, 70), natoms=3, numax=9, nbands=9)
    hd = api.Handle(0)
    hd.set_support_radius(5.3)
    for prec in ("fp64", "ff64"):
        got = api.project(torch.from_numpy(psi).cuda(), pos, sig, 9, 64, h, True, prec=prec, handle=hd)
        ref = oracle.project(grid, h, True, psi, pos, sig, 9, 64, rprj=5.3)
        assert_coeff_close(got.cpu().numpy(), ref, TOL_FP64)
    hd.close()


def test_sphere_nonlocal_ff64():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, _ = _case(1502, nbands=24)
    numax, cube, R = 5, 32, 2.6
    N = oracle.nstates(numax)
    rng = np.random.default_rng(1503)
    D = rng.uniform(-1, 1, size=(len(pos), N, N))
    hd = api.Handle(0)
    hd.set_support_radius(R)
    out = torch.zeros(psi.shape, dtype=torch.float64, device="cuda")
    api.apply_nonlocal(torch.from_numpy(psi).cuda(), out, torch.from_numpy(D).cuda(), pos, sig, numax, cube, h, True,
                       prec="ff64", handle=hd)
    cref = oracle.project(grid, h, True, psi, pos, sig, numax, cube, rprj=R)
    ref = oracle.add(grid, h, True, np.zeros_like(psi), pos, sig, numax, cube, np.einsum("akl,alb->akb", D, cref),
                     rprj=R)
    assert rel_norm(out.cpu().numpy(), ref) <= TOL_FP64
    hd.close()


def test_sphere_stored_projectors_match_sho():
    """The stored-projector baseline built with the same sphere gives the SHO sphere projection."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, c = _case(1504, natoms=4, numax=3, nbands=16, periodic=False)
    hd = api.Handle(0)
    hd.set_support_radius(2.2)
    psi_d = torch.from_numpy(psi).cuda()
    proj = api.usu_build(pos, sig, 3, 32, grid, h, False, handle=hd)
    got = api.usu_project(psi_d, proj, pos, sig, 3, 32, h, False, handle=hd).cpu().numpy()
    ref = oracle.project(grid, h, False, psi, pos, sig, 3, 32, rprj=2.2)
    assert_coeff_close(got, ref, TOL_FP64)
    out = torch.zeros_like(psi_d)
    api.usu_add(out, torch.from_numpy(c).cuda(), proj, pos, sig, 3, 32, h, False, handle=hd)
    ref2 = oracle.add(grid, h, False, np.zeros_like(psi), pos, sig, 3, 32, c, rprj=2.2)
    assert rel_norm(out.cpu().numpy(), ref2) <= TOL_FP64
    hd.close()


def test_sphere_refused_where_not_implemented():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import ShoError, api
    hd = api.Handle(0)
    hd.set_support_radius(2.0)
    psi = torch.zeros((40, 40, 40, 8), dtype=torch.float32, device="cuda")
    for prec in ("fp32", "tf32", "bf16"):
        with pytest.raises(ShoError, match="DTYPE"):
            api.project(psi, np.array([[3.0, 3.0, 3.0]]), [0.7], 3, 16, 0.2, True, prec=prec, handle=hd)
    z = torch.zeros((40, 40, 40, 2), dtype=torch.complex128, device="cuda")
    with pytest.raises(ShoError, match="DTYPE"):
        api.project_bloch(z, [0.1, 0.2, 0.3], np.array([[3.0, 3.0, 3.0]]), [0.7], 3, 16, 0.2, handle=hd)
    with pytest.raises(ShoError, match="ARG"):
        hd.set_support_radius(-1.0)
    hd.close()
