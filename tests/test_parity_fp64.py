"""FP64 parity of the CUDA path against the oracle (GPU).

Small and medium cases run the full oracle; the 96^3 / 64-atom / 128-band production case checks
sampled atoms (projection) and sampled grid points (expansion) at full size, in the launch
configuration the benchmark uses.  Bar: 1e-12 relative (norm-wise per atom and max-wise)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, assert_coeff_close, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _api():
    from paper_1905_00480_gb300 import api
    return api


def _case(grid, h, periodic, natoms, numax, cube, nbands, seed, sigma_range=(0.5, 1.0)):
    rng = np.random.default_rng(seed)
    box = tuple(n * h for n in grid)
    pos, sig = workloads.random_atoms(rng, natoms, box, periodic, min_sep=0.5, sigma_range=sigma_range)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return pos, sig, psi, c


def _check_all(grid, h, periodic, pos, sig, psi, c, numax, cube, forces=True):
    require_gpu()
    api = _api()
    got = api.project(_t(psi), pos, sig, numax, cube, h, periodic, prec="fp64").cpu().numpy()
    ref = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube)
    assert_coeff_close(got, ref, TOL_FP64)
    out = _t(psi)
    api.add(out, _t(c), pos, sig, numax, cube, h, periodic, prec="fp64")
    ref2 = oracle.add(grid, h, periodic, psi, pos, sig, numax, cube, c)
    d_got, d_ref = out.cpu().numpy() - psi, ref2 - psi
    assert rel_norm(d_got, d_ref) <= TOL_FP64
    assert rel_max(d_got, d_ref) <= TOL_FP64
    if forces:
        f = api.forces(_t(psi), _t(c), pos, sig, numax, cube, h, periodic, prec="fp64").cpu().numpy()
        ref3 = oracle.forces(grid, h, periodic, psi, pos, sig, numax, cube, c)
        assert rel_max(f, ref3) <= TOL_FP64


def test_tiny_config_full():
    w = workloads.WORKLOADS["tiny"]
    pos, sig = workloads.atoms(w)
    psi = workloads.psi_host(w)
    c = workloads.coeff_host(w, oracle.nstates(w.numax))
    _check_all(w.grid, w.h, w.periodic, pos, sig, psi, c, w.numax, w.cube)


@pytest.mark.parametrize("periodic", [True, False])
def test_medium_ragged(periodic):
    """Several cubes per axis, a ragged band tile (45 bands = 32 + 13), uneven grid extents."""
    grid, h = (40, 36, 44), 0.2
    pos, sig, psi, c = _case(grid, h, periodic, 7, 4, 16, 45, seed=21)
    _check_all(grid, h, periodic, pos, sig, psi, c, 4, 16)


@pytest.mark.parametrize("numax", [0, 1, 9])
def test_numax_extremes(numax):
    grid, h = (24, 24, 24), 0.25
    pos, sig, psi, c = _case(grid, h, True, 3, numax, 16, 33, seed=30 + numax)
    _check_all(grid, h, True, pos, sig, psi, c, numax, 16)


@pytest.mark.parametrize("cube", [8, 24, 64])
def test_cube_sizes(cube):
    grid, h = (64, 64, 64) if cube == 64 else (32, 40, 36), 0.2
    pos, sig, psi, c = _case(grid, h, True, 2, 3, cube, 8, seed=40 + cube)
    _check_all(grid, h, True, pos, sig, psi, c, 3, cube)


def test_single_band_and_edge_positions():
    """B = 1; an atom exactly on a grid point (X/h integral), one outside [0, L) (periodic wrap through the
    cube origin), one near a corner of a non-periodic grid (clipped cube)."""
    grid, h = (32, 32, 32), 0.25
    pos = np.array([[4.0, 2.5, 6.0], [-1.13, 9.61, 3.3], [0.2, 7.7, 0.4]])
    sig = np.array([0.8, 0.6, 0.9])
    rng = np.random.default_rng(50)
    psi = rng.standard_normal((32, 32, 32, 1))
    c = rng.standard_normal((3, oracle.nstates(4), 1))
    _check_all(grid, h, True, pos, sig, psi, c, 4, 16)
    _check_all(grid, h, False, pos, sig, psi, c, 4, 16)


def test_empty_inputs_are_noops():
    require_gpu()
    import torch
    api = _api()
    psi = torch.zeros((16, 16, 16, 4), dtype=torch.float64, device="cuda")
    c = api.project(psi, np.zeros((0, 3)), np.zeros(0), 3, 16, 0.25, True)
    assert tuple(c.shape) == (0, 20, 4)
    api.add(psi, torch.zeros((0, 20, 4), dtype=torch.float64, device="cuda"), np.zeros((0, 3)), np.zeros(0), 3, 16,
            0.25, True)
    assert float(psi.abs().max()) == 0.0


def test_adjoint_identity_gpu():
    require_gpu()
    api = _api()
    grid, h = (36, 36, 36), 0.2
    pos, sig, psi, c = _case(grid, h, True, 5, 5, 32, 40, seed=60)
    lhs = float((api.project(_t(psi), pos, sig, 5, 32, h, True).cpu().numpy() * c).sum())
    z = _t(np.zeros_like(psi))
    api.add(z, _t(c), pos, sig, 5, 32, h, True)
    rhs = h ** 3 * float((psi * z.cpu().numpy()).sum())
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_deterministic_bitwise():
    require_gpu()
    api = _api()
    grid, h = (40, 40, 40), 0.2
    pos, sig, psi, c = _case(grid, h, True, 9, 5, 32, 64, seed=70)
    a1 = api.project(_t(psi), pos, sig, 5, 32, h, True).cpu().numpy()
    a2 = api.project(_t(psi), pos, sig, 5, 32, h, True).cpu().numpy()
    assert np.array_equal(a1, a2)
    p1, p2 = _t(psi), _t(psi)
    api.add(p1, _t(c), pos, sig, 5, 32, h, True)
    api.add(p2, _t(c), pos, sig, 5, 32, h, True)
    assert np.array_equal(p1.cpu().numpy(), p2.cpu().numpy())


def test_production_size_sampled():
    """96^3 periodic grid, 64 atoms, numax 5, cube 32, 128 bands (the benchmark workload): projection
    checked on 6 sampled atoms, expansion on 400 sampled grid points, both against the oracle."""
    require_gpu()
    import torch
    api = _api()
    w = workloads.WORKLOADS["c96"]
    pos, sig = workloads.atoms(w)
    psi = workloads.psi_host(w)
    N = oracle.nstates(w.numax)
    c_in = workloads.coeff_host(w, N)
    psi_d = _t(psi)
    got = api.project(psi_d, pos, sig, w.numax, w.cube, w.h, w.periodic).cpu().numpy()
    rng = np.random.default_rng(99)
    sel = np.sort(rng.choice(w.natoms, size=6, replace=False))
    ref = oracle.project(w.grid, w.h, w.periodic, psi, pos[sel], sig[sel], w.numax, w.cube)
    assert_coeff_close(got[sel], ref, TOL_FP64)
    api.add(psi_d, _t(c_in), pos, sig, w.numax, w.cube, w.h, w.periodic)
    out = psi_d.cpu().numpy().reshape(-1, w.nbands)
    pts = rng.choice(out.shape[0], size=400, replace=False)
    ref_pts = oracle.expand_points(w.grid, w.h, w.periodic, pos, sig, w.numax, w.cube, c_in, pts)
    d_got = out[pts] - psi.reshape(-1, w.nbands)[pts]
    assert rel_norm(d_got, ref_pts) <= TOL_FP64
    assert rel_max(d_got, ref_pts) <= TOL_FP64
    del psi_d
    torch.cuda.empty_cache()
