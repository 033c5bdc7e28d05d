"""sho_add_scaled: psi = (0 if overwrite else psi) + alpha E c with the factor applied inside the
kernels (GPU).  alpha = h^3 is the adjoint of the projection in the plain grid inner product (Sec. 3.2,
steps 1 and 3), the gradient the autograd backward needs."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp64": TOL_FP64, "ff64": TOL_FP64, "fp32": 2e-6, "tf32": 2e-3, "split_fp16": 1e-5}


def _case(seed, grid=(40, 36, 44), natoms=6, nbands=40, numax=5):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * 0.2 for n in grid), True, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return grid, pos, sig, psi, c, numax


@pytest.mark.parametrize("prec", ["fp64", "ff64", "fp32", "tf32", "split_fp16"])
def test_scaled_overwrite_matches_oracle(prec):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, c, numax = _case(1201)
    h, cube = 0.2, 32
    f64 = prec in ("fp64", "ff64")
    tdt = torch.float64 if f64 else torch.float32
    c_d = torch.from_numpy(c).cuda().to(tdt)
    out = torch.from_numpy(psi).cuda().to(tdt)       # garbage to be overwritten
    api.add(out, c_d, pos, sig, numax, cube, h, True, prec=prec, alpha=h ** 3, overwrite=True)
    ref = h ** 3 * oracle.add(grid, h, True, np.zeros_like(psi), pos, sig, numax, cube, c_d.double().cpu().numpy())
    got = out.double().cpu().numpy()
    assert rel_norm(got, ref) <= TOL[prec]
    assert rel_max(got, ref) <= 2 * TOL[prec]
    # points outside every cube were cleared
    cover = oracle.add(grid, h, True, np.zeros_like(psi), pos, sig, numax, cube, np.ones_like(c)) != 0
    assert float(np.abs(got[~cover]).max(initial=0.0)) == 0.0


@pytest.mark.parametrize("prec", ["fp64", "fp32"])
def test_scaled_accumulate_and_unit_alpha_is_sho_add(prec):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, c, numax = _case(1202, numax=4)
    h, cube = 0.2, 16
    tdt = torch.float64 if prec == "fp64" else torch.float32
    c_d = torch.from_numpy(c).cuda().to(tdt)
    p1 = torch.from_numpy(psi).cuda().to(tdt)
    p2 = p1.clone()
    api.add(p1, c_d, pos, sig, numax, cube, h, True, prec=prec)
    api.add(p2, c_d, pos, sig, numax, cube, h, True, prec=prec, alpha=1.0 + 0.0, overwrite=False)
    assert torch.equal(p1, p2)
    # the scaled entry point itself with alpha = 1 (not routed to sho_add by the binding)
    from paper_1905_00480_gb300 import _native as N
    p3 = torch.from_numpy(psi).cuda().to(tdt)
    g = api._grid(p3, h, True)
    pos_h, sig_h = np.ascontiguousarray(pos), np.ascontiguousarray(sig)
    dt = N.DTYPES["f64" if prec == "fp64" else "f32"]
    st = N.lib().sho_add_scaled(api.default_handle(0).ptr, api.ctypes.byref(g), 1.0, 0,
                                api.ctypes.c_void_p(c_d.data_ptr()), dt, psi.shape[3], len(pos), api._dp(pos_h),
                                api._dp(sig_h), numax, cube, N.PRECS[prec], api.ctypes.c_void_p(p3.data_ptr()), dt,
                                api._stream_ptr(p3, None))
    assert st == 0
    assert torch.equal(p1, p3)
    # accumulate with alpha = -0.5: psi - 0.5 E c
    p4 = torch.from_numpy(psi).cuda().to(tdt)
    api.add(p4, c_d, pos, sig, numax, cube, h, True, prec=prec, alpha=-0.5)
    ref = oracle.add(grid, h, True, np.zeros_like(psi), pos, sig, numax, cube, c_d.double().cpu().numpy())
    d = p4.double().cpu().numpy() - torch.from_numpy(psi).to(tdt).double().numpy()
    assert rel_norm(d, -0.5 * ref) <= TOL[prec]


def test_overwrite_without_atoms_clears_and_bad_alpha_is_rejected():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import ShoError, api
    psi = torch.ones((16, 16, 16, 4), dtype=torch.float64, device="cuda")
    api.add(psi, torch.zeros((0, 20, 4), dtype=torch.float64, device="cuda"), np.zeros((0, 3)), np.zeros(0), 3, 16,
            0.25, True, alpha=2.0, overwrite=True)
    assert float(psi.abs().max()) == 0.0
    with pytest.raises(ShoError, match="ARG"):
        api.add(psi, torch.zeros((1, 20, 4), dtype=torch.float64, device="cuda"), np.ones((1, 3)), np.ones(1), 3, 16,
                0.25, True, alpha=float("nan"))
