"""Non-local action hpsi += sum_a |k> D_a <k|psi> (Sec. 3.2 steps 1-3 with the SHO basis of Sec. 3.5)
against the oracle: oracle projection, the matrix product as a library step, oracle expansion (GPU)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, TOL_FP64, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _case(seed, grid=(40, 36, 44), h=0.2, natoms=6, numax=5, nbands=40, periodic=True):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * h for n in grid), periodic, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    hpsi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    N = oracle.nstates(numax)
    D = rng.uniform(-1, 1, size=(natoms, N, N))
    D = 0.5 * (D + D.transpose(0, 2, 1))           # symmetric, as an atomic Hamiltonian block
    return grid, h, pos, sig, psi, hpsi, D


def _reference(grid, h, periodic, pos, sig, psi, hpsi, D, numax, cube):
    c = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube)
    d = np.einsum("akl,alb->akb", D, c)
    return oracle.add(grid, h, periodic, hpsi, pos, sig, numax, cube, d)


@pytest.mark.parametrize("prec,storage,tol", [("fp64", "f64", TOL_FP64), ("ff64", "f64", TOL_FP64),
                                              ("fp32", "f32", 10 * TOL_FP32), ("tf32", "f32", 1e-2),
                                              ("3xtf32", "f32", 1e-5)])
@pytest.mark.parametrize("periodic", [True, False])
def test_nonlocal_action(prec, storage, tol, periodic):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, hpsi, D = _case(700, periodic=periodic)
    tdt = {"f64": torch.float64, "f32": torch.float32}[storage]
    cdt = torch.float64 if prec in ("fp64", "ff64") else torch.float32
    psi_d = torch.from_numpy(psi).cuda().to(tdt)
    hpsi_d = torch.from_numpy(hpsi).cuda().to(tdt)
    D_d = torch.from_numpy(D).cuda().to(cdt)
    psi_r, hpsi_r = psi_d.double().cpu().numpy(), hpsi_d.double().cpu().numpy()
    api.apply_nonlocal(psi_d, hpsi_d, D_d, pos, sig, 5, 32, h, periodic, prec=prec)
    ref = _reference(grid, h, periodic, pos, sig, psi_r, hpsi_r, D_d.double().cpu().numpy(), 5, 32)
    assert rel_norm(hpsi_d.double().cpu().numpy() - hpsi_r, ref - hpsi_r) <= tol


def test_nonlocal_identity_D_is_projector():
    """With D = identity the action is E P psi, the truncated SHO projector of Sec. 2.5 (times h^3 of
    the quadrature): applied to a sampled SHO state on a wide, fine cube it reproduces the state."""
    require_gpu()
    import math
    import torch
    from paper_1905_00480_gb300 import api
    h, sigma, numax, cube = 0.2, 0.8, 3, 64
    grid = (64, 64, 64)
    X = np.array([[6.37, 6.52, 6.18]])
    xs = np.arange(64) * h

    def phi(n, u):
        from scipy import special
        xi = u / sigma
        return special.eval_hermite(n, xi) * np.exp(-0.5 * xi * xi) / math.sqrt(sigma * math.sqrt(math.pi) * 2.0 ** n * math.factorial(n))

    state = np.einsum("z,y,x->zyx", phi(1, xs - X[0, 2]), phi(0, xs - X[0, 1]), phi(2, xs - X[0, 0]))[..., None]
    psi_d = torch.from_numpy(state).cuda()
    out = torch.zeros_like(psi_d)
    N = oracle.nstates(numax)
    D = torch.eye(N, dtype=torch.float64, device="cuda")[None].contiguous()
    api.apply_nonlocal(psi_d, out, D, X, [sigma], numax, cube, h, False, prec="ff64")
    assert rel_norm(out.cpu().numpy(), state) < 1e-11
