"""Device checks (sho_set_device_checks), the memory-checker stand-in of the FP64 and FP64-accurate
kernels (GPU).

With the checks on, the projection, expansion and forces of both forms give bit for bit the results of
the unchecked kernels and report nothing.  With psi's extent declared smaller than the buffer
(sho_fault_check_extent: every access still lands inside the real buffer, the checked ones beyond the
declared extent are skipped), each call reports SHO_ERR_DEVICE through sho_sync, and the next call with
the real extent is clean and matches the oracle."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, assert_coeff_close, rel_norm, require_gpu

pytestmark = pytest.mark.gpu

ERR_DEVICE = -9


def _case(seed=930, grid=(40, 36, 44), natoms=5, nbands=32, numax=4):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * 0.2 for n in grid), True, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return grid, pos, sig, psi, c, numax


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _run(api, hd, grid, pos, sig, psi, c, numax, prec):
    got_c = api.project(_t(psi), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd).cpu().numpy()
    out = _t(psi)
    api.add(out, _t(c), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd)
    f = api.forces(_t(psi), _t(c), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd).cpu().numpy()
    return got_c, out.cpu().numpy(), f


@pytest.mark.parametrize("prec", ["fp64", "ff64"])
def test_checked_kernels_match_unchecked_bit_for_bit(prec):
    require_gpu()
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, c, numax = _case()
    plain = api.Handle(0)
    plain.set_expand_kernel("mma_sync")  # the float-float kernels, the ones the checked mode runs
    plain.set_project_kernel("mma_sync")
    ref = _run(api, plain, grid, pos, sig, psi, c, numax, prec)
    assert N.lib().sho_sync(plain.ptr) == 0
    plain.close()
    hd = api.Handle(0)
    hd.set_device_checks(True)
    got = _run(api, hd, grid, pos, sig, psi, c, numax, prec)
    assert N.lib().sho_sync(hd.ptr) == 0
    hd.close()
    for a, b in zip(got, ref):
        assert np.array_equal(a, b)
    assert_coeff_close(got[0], oracle.project(grid, 0.2, True, psi, pos, sig, numax, 16), TOL_FP64)


@pytest.mark.parametrize("prec", ["fp64", "ff64"])
@pytest.mark.parametrize("op", ["project", "add"])
def test_declared_extent_violation_is_reported_and_next_call_is_clean(prec, op):
    require_gpu()
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, c, numax = _case(seed=931)
    hd = api.Handle(0)
    hd.set_device_checks(True)
    L = N.lib()
    assert L.sho_fault_check_extent(hd.ptr, psi.size // 2) == 0   # half of psi's real extent
    if op == "project":
        api.project(_t(psi), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd)
    else:
        out = _t(psi)
        api.add(out, _t(c), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd)
        # the checked stores above the declared extent were skipped: that part of psi is unchanged there
        back = out.cpu().numpy().reshape(-1)
        tail = slice(psi.size // 2, None)
        assert np.array_equal(back[tail], psi.reshape(-1)[tail])
    assert L.sho_sync(hd.ptr) == ERR_DEVICE
    assert L.sho_sync(hd.ptr) == 0
    assert L.sho_fault_check_extent(hd.ptr, -1) == 0
    if op == "project":
        got = api.project(_t(psi), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd).cpu().numpy()
        assert L.sho_sync(hd.ptr) == 0
        assert_coeff_close(got, oracle.project(grid, 0.2, True, psi, pos, sig, numax, 16), TOL_FP64)
    else:
        out = _t(psi)
        api.add(out, _t(c), pos, sig, numax, 16, 0.2, True, prec=prec, handle=hd)
        assert L.sho_sync(hd.ptr) == 0
        ref = oracle.add(grid, 0.2, True, psi, pos, sig, numax, 16, c)
        assert rel_norm(out.cpu().numpy() - psi, ref - psi) <= TOL_FP64
    hd.close()
