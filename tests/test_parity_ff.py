"""FP64-accurate float-float form (SHO_P_FF64) against the FP64 oracle (GPU).

The x-pass runs as float-float dot products (psi and the 1D functions carried to ~48 bits, products
error-free, sums compensated); everything else is FP64.  Expected norm-wise error ~1e-13; the bar is
the FP64 one, 1e-12."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, assert_coeff_close, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _check(grid, h, periodic, pos, sig, psi, c, numax, cube, forces=True):
    require_gpu()
    from paper_1905_00480_gb300 import api
    got = api.project(_t(psi), pos, sig, numax, cube, h, periodic, prec="ff64").cpu().numpy()
    ref = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube)
    assert_coeff_close(got, ref, TOL_FP64)
    out = _t(psi)
    api.add(out, _t(c), pos, sig, numax, cube, h, periodic, prec="ff64")
    ref2 = oracle.add(grid, h, periodic, psi, pos, sig, numax, cube, c)
    assert rel_norm(out.cpu().numpy() - psi, ref2 - psi) <= TOL_FP64
    assert rel_max(out.cpu().numpy() - psi, ref2 - psi) <= TOL_FP64
    if forces:
        f = api.forces(_t(psi), _t(c), pos, sig, numax, cube, h, periodic, prec="ff64").cpu().numpy()
        ref3 = oracle.forces(grid, h, periodic, psi, pos, sig, numax, cube, c)
        assert rel_max(f, ref3) <= TOL_FP64


def test_ff_tiny():
    w = workloads.WORKLOADS["tiny"]
    pos, sig = workloads.atoms(w)
    _check(w.grid, w.h, w.periodic, pos, sig, workloads.psi_host(w), workloads.coeff_host(w, oracle.nstates(w.numax)),
           w.numax, w.cube)


@pytest.mark.parametrize("periodic", [True, False])
@pytest.mark.parametrize("numax", [0, 4, 9])
def test_ff_medium_ragged(periodic, numax):
    rng = np.random.default_rng(600 + numax)
    grid, h = (40, 36, 44), 0.2
    pos, sig = workloads.random_atoms(rng, 6, tuple(n * h for n in grid), periodic, min_sep=0.5)
    psi = rng.standard_normal((44, 36, 40, 45))
    c = rng.standard_normal((6, oracle.nstates(numax), 45))
    _check(grid, h, periodic, pos, sig, psi, c, numax, 16)


def test_ff_wide_dynamic_range():
    """psi spanning 1e-20 .. 1e20 in magnitude (inside the FP32 normal range the form requires) for the
    projection; coefficients of 1e10 expanded into a zero grid (an update added to values of 1e20
    would lose its own digits to the rounding of the sum on both sides)."""
    require_gpu()
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(610)
    grid, h = (32, 32, 32), 0.25
    pos, sig = workloads.random_atoms(rng, 3, (8.0, 8.0, 8.0), True, min_sep=1.0)
    psi = rng.standard_normal((32, 32, 32, 8)) * 10.0 ** rng.uniform(-20, 20, size=(32, 32, 32, 8))
    got = api.project(_t(psi), pos, sig, 5, 32, h, True, prec="ff64").cpu().numpy()
    assert_coeff_close(got, oracle.project(grid, h, True, psi, pos, sig, 5, 32), TOL_FP64)
    c = rng.standard_normal((3, oracle.nstates(5), 8)) * 1e10
    out = _t(np.zeros_like(psi))
    api.add(out, _t(c), pos, sig, 5, 32, h, True, prec="ff64")
    ref = oracle.add(grid, h, True, np.zeros_like(psi), pos, sig, 5, 32, c)
    assert rel_norm(out.cpu().numpy(), ref) <= TOL_FP64


def test_ff_production_size_sampled():
    require_gpu()
    from paper_1905_00480_gb300 import api
    w = workloads.WORKLOADS["c96"]
    pos, sig = workloads.atoms(w)
    psi = workloads.psi_host(w)
    c_in = workloads.coeff_host(w, oracle.nstates(w.numax))
    psi_d = _t(psi)
    got = api.project(psi_d, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="ff64").cpu().numpy()
    sel = np.array([3, 17, 41])
    ref = oracle.project(w.grid, w.h, w.periodic, psi, pos[sel], sig[sel], w.numax, w.cube)
    assert_coeff_close(got[sel], ref, TOL_FP64)
    api.add(psi_d, _t(c_in), pos, sig, w.numax, w.cube, w.h, w.periodic, prec="ff64")
    out = psi_d.cpu().numpy().reshape(-1, w.nbands)
    pts = np.random.default_rng(1).choice(out.shape[0], size=300, replace=False)
    ref_pts = oracle.expand_points(w.grid, w.h, w.periodic, pos, sig, w.numax, w.cube, c_in, pts)
    assert rel_norm(out[pts] - psi.reshape(-1, w.nbands)[pts], ref_pts) <= TOL_FP64
