"""Non-local action hpsi += sum_a |k> D_a <k|psi> (Sec. 3.2 steps 1-3 with the SHO basis of Sec. 3.5)
against the oracle: oracle projection, the matrix product, oracle expansion (GPU).

The library fuses the action: the projection stops at its per-plane sums (FP64-accurate form, plane sweep)
or its coefficients (other paths), and the expansion's z-pass kernel finishes the projection, multiplies
by D and expands with c and d in shared memory.  The cases cover every path into that kernel: FP64
clusters and per-atom FP32 kernels (coefficient input), FF64 and plane sweep (per-plane-sum input, FP32
and BF16 storage), numax 8-9 (shared-memory columns beyond 48 KB)."""
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


@pytest.mark.parametrize("prec,storage,numax,tol", [
    ("split_fp16", "f32", 5, 1e-5), ("bf16", "f32", 5, 3e-2),              # plane sweep, tensor forms
    ("tf32", "bf16", 5, 1e-2), ("fp32", "bf16", 7, 10 * TOL_FP32),         # plane sweep over BF16 rows
    ("fp32", "f32", 8, 10 * TOL_FP32),                                     # per-atom kernels (numax 8)
    ("ff64", "f64", 9, TOL_FP64), ("fp64", "f64", 9, TOL_FP64)])           # 220 states
def test_nonlocal_paths(prec, storage, numax, tol):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, hpsi, D = _case(701 + numax, numax=numax, nbands=48, natoms=5)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[storage]
    cdt = torch.float64 if prec in ("fp64", "ff64") else torch.float32
    psi_d = torch.from_numpy(psi).cuda().to(tdt)
    hpsi_d = torch.zeros_like(psi_d)
    D_d = torch.from_numpy(D).cuda().to(cdt)
    api.apply_nonlocal(psi_d, hpsi_d, D_d, pos, sig, numax, 32, h, True, prec=prec)
    ref = _reference(grid, h, True, pos, sig, psi_d.double().cpu().numpy(), np.zeros(psi.shape),
                     D_d.double().cpu().numpy(), numax, 32)
    tol_store = 2.0 ** -8 if storage == "bf16" else 0.0    # the result is rounded to BF16 on store
    assert rel_norm(hpsi_d.double().cpu().numpy(), ref) <= tol + tol_store


@pytest.mark.parametrize("prec", ["ff64", "tf32"])
def test_fused_action_matches_composed_calls(prec):
    """The fused action equals projection, D c and expansion run as separate library calls (the same
    arithmetic up to the order of the D product's sums)."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, pos, sig, psi, hpsi, D = _case(720)
    cdt = torch.float64 if prec == "ff64" else torch.float32
    psi_d = torch.from_numpy(psi).cuda().to(cdt)
    D_d = torch.from_numpy(D).cuda().to(cdt)
    fused = torch.zeros_like(psi_d)
    api.apply_nonlocal(psi_d, fused, D_d, pos, sig, 5, 32, h, True, prec=prec)
    c = api.project(psi_d, pos, sig, 5, 32, h, True, prec=prec)
    d = torch.einsum("akl,alb->akb", D_d.double(), c.double()).to(cdt).contiguous()
    composed = torch.zeros_like(psi_d)
    api.add(composed, d, pos, sig, 5, 32, h, True, prec=prec)
    tol = 1e-13 if prec == "ff64" else 1e-5
    assert rel_norm(fused.double().cpu().numpy(), composed.double().cpu().numpy()) <= tol
