"""Failure detection without a GPU fault (GPU).

Every injected failure here ends by itself and leaves the context usable:
  * the plane-sweep projection's bounded mbarrier waits run out because the producer warp stops issuing
    rows (sho_fault_stop_rows) under a short wait limit (sho_fault_wait_limit); the kernel records the
    timeout, returns, and sho_sync reports SHO_ERR_TIMEOUT; the next normal call is correct;
  * the FP64-accurate (float-float) form meets inputs outside the float-pair range and sho_sync reports
    SHO_ERR_DEVICE, while the native FP64 form computes the same data exactly;
  * a served request meets the same injected pipeline failure, and its status (not a silent success)
    comes back through sho_wait_status;
  * a request held by the scheduler (sho_fault_hold, a stuck request as the host sees it) times out for
    its waiter while other systems keep being served, queued requests behind it can be cancelled
    (sho_cancel), and it completes once released.
"""
import ctypes
import threading

import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, TOL_FP64, assert_coeff_close, rel_norm, require_gpu

pytestmark = pytest.mark.gpu

SHORT_WAIT = 200_000      # SM clock cycles, ~0.1 ms: far below the ~2 s default
ERR_TIMEOUT, ERR_DEVICE, ERR_STATE, ERR_CANCELLED = -8, -9, -11, -12


def _fp32_case(seed=901, grid=(48, 48, 48), natoms=10, nbands=64, numax=5):
    import torch
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * 0.2 for n in grid), True, min_sep=1.0)
    psi = torch.from_numpy(rng.standard_normal((grid[2], grid[1], grid[0], nbands)).astype(np.float32)).cuda()
    return grid, pos, sig, psi, numax


def test_plane_sweep_bounded_wait_runs_out_and_next_call_is_clean():
    require_gpu()
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, numax = _fp32_case()
    assert api.project_path(psi, numax, 32, 0.2, True, prec="fp32") == "plane"
    hd = api.Handle(0)
    L = N.lib()
    assert L.sho_fault_wait_limit(hd.ptr, SHORT_WAIT) == 0
    assert L.sho_fault_stop_rows(hd.ptr, 1) == 0
    api.project(psi, pos, sig, numax, 32, 0.2, True, prec="fp32", handle=hd)
    assert L.sho_sync(hd.ptr) == ERR_TIMEOUT
    assert L.sho_sync(hd.ptr) == 0                     # the status word was cleared
    assert L.sho_fault_wait_limit(hd.ptr, 0) == 0
    assert L.sho_fault_stop_rows(hd.ptr, -1) == 0
    got = api.project(psi, pos, sig, numax, 32, 0.2, True, prec="fp32", handle=hd)
    assert L.sho_sync(hd.ptr) == 0
    ref = oracle.project(grid, 0.2, True, psi.double().cpu().numpy(), pos, sig, numax, 32)
    assert_coeff_close(got.double().cpu().numpy(), ref, TOL_FP32)
    assert L.sho_fault_wait_limit(hd.ptr, -5) == -1    # SHO_ERR_ARG
    hd.close()


def _f64_case(seed=902, grid=(40, 36, 44), natoms=5, nbands=33, numax=4):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * 0.2 for n in grid), True, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return grid, pos, sig, psi, c, numax


@pytest.mark.parametrize("scale", [1e-300, 1e300])
def test_ff64_range_guard_projection(scale):
    """psi far outside the float exponent range: FF64 reports SHO_ERR_DEVICE; FP64 is exact."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, _, numax = _f64_case()
    bad = psi * scale
    hd = api.Handle(0)
    api.project(torch.from_numpy(bad).cuda(), pos, sig, numax, 16, 0.2, True, prec="ff64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == ERR_DEVICE
    got = api.project(torch.from_numpy(bad).cuda(), pos, sig, numax, 16, 0.2, True, prec="fp64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == 0
    ref = oracle.project(grid, 0.2, True, bad, pos, sig, numax, 16)
    assert_coeff_close(got.cpu().numpy() / scale, ref / scale, TOL_FP64)   # rescaled: norms stay finite
    # exact zeros are inside the range: a band of zeros is not flagged and the result is FP64-accurate
    zeros = psi.copy()
    zeros[:, :, :, 0] = 0.0
    got = api.project(torch.from_numpy(zeros).cuda(), pos, sig, numax, 16, 0.2, True, prec="ff64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == 0
    ref = oracle.project(grid, 0.2, True, zeros, pos, sig, numax, 16)
    assert_coeff_close(got.cpu().numpy(), ref, TOL_FP64)
    hd.close()


def test_ff64_range_guard_single_covered_value():
    """A single tiny value at a grid point inside an atom's cube is detected."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, _, numax = _f64_case(seed=903)
    o = np.floor(pos[0] / 0.2).astype(int)   # a grid point next to atom 0 lies in its cube
    mixed = psi.copy()
    mixed[o[2] % grid[2], o[1] % grid[1], o[0] % grid[0], 2] = 3e-39   # below 2^-126
    hd = api.Handle(0)
    api.project(torch.from_numpy(mixed).cuda(), pos, sig, numax, 16, 0.2, True, prec="ff64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == ERR_DEVICE
    hd.close()


def test_ff64_range_guard_expansion():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    grid, pos, sig, psi, c, numax = _f64_case(seed=904)
    hd = api.Handle(0)
    out = torch.zeros(psi.shape, dtype=torch.float64, device="cuda")
    api.add(out, torch.from_numpy(c * 1e300).cuda(), pos, sig, numax, 16, 0.2, True, prec="ff64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == ERR_DEVICE
    out.zero_()
    api.add(out, torch.from_numpy(c * 1e300).cuda(), pos, sig, numax, 16, 0.2, True, prec="fp64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == 0
    ref = oracle.add(grid, 0.2, True, np.zeros_like(psi), pos, sig, numax, 16, c * 1e300)
    assert rel_norm(out.cpu().numpy() / 1e300, ref / 1e300) <= TOL_FP64   # rescaled: norms stay finite
    out.zero_()
    api.add(out, torch.from_numpy(c).cuda(), pos, sig, numax, 16, 0.2, True, prec="ff64", handle=hd)
    assert N.lib().sho_sync(hd.ptr) == 0
    ref = oracle.add(grid, 0.2, True, np.zeros_like(psi), pos, sig, numax, 16, c)
    assert rel_norm(out.cpu().numpy(), ref) <= TOL_FP64
    hd.close()


def test_served_request_reports_device_timeout():
    require_gpu()
    from paper_1905_00480_gb300.serve import Server
    grid, pos, sig, psi, numax = _fp32_case(seed=905)
    with Server(0, budget_bytes=4 << 30, slots=2) as srv:
        sid = srv.register(psi, pos, sig, numax, 32, 0.2)
        srv.fault_pipeline(SHORT_WAIT, 1)
        assert srv.wait(srv.submit(sid, "project", "fp32"), 60000) == ERR_TIMEOUT
        st = srv.stats()
        assert st["failed"] == 1 and st["completed"] == 1
        srv.fault_pipeline(0, -1)
        assert srv.wait(srv.submit(sid, "project", "fp32"), 60000) == 0
        _, c = srv.read(sid, psi=False)
        srv.unregister(sid)
    ref = oracle.project(grid, 0.2, True, psi.double().cpu().numpy(), pos, sig, numax, 32)
    assert_coeff_close(c.double().numpy(), ref, TOL_FP32)


def test_served_ff64_out_of_range_is_reported():
    require_gpu()
    import torch
    from paper_1905_00480_gb300.serve import Server
    grid, pos, sig, psi, _, numax = _f64_case(seed=906)
    with Server(0, budget_bytes=4 << 30, slots=2) as srv:
        sid = srv.register(torch.from_numpy(psi * 1e300).cuda(), pos, sig, numax, 16, 0.2)
        assert srv.wait(srv.submit(sid, "project", "ff64"), 60000) == ERR_DEVICE
        assert srv.wait(srv.submit(sid, "project", "fp64"), 60000) == 0
        srv.unregister(sid)


def test_stuck_request_cancel_and_release():
    require_gpu()
    from paper_1905_00480_gb300 import api
    from paper_1905_00480_gb300.serve import Server
    ga, pa, sa, psia, nua = _fp32_case(seed=907)
    gb, pb, sb, psib, nub = _fp32_case(seed=908, grid=(40, 40, 40), natoms=6, nbands=32, numax=3)
    with Server(0, budget_bytes=4 << 30, slots=2) as srv:
        A = srv.register(psia, pa, sa, nua, 32, 0.2)
        B = srv.register(psib, pb, sb, nub, 32, 0.2)
        srv.fault_hold(A, True)
        t1 = srv.submit(A, "project", "fp32")
        with pytest.raises(TimeoutError):
            srv.wait(t1, 200)                          # stuck: its waiter's bounded wait runs out
        t3 = srv.submit(A, "expand", "fp32")           # queued behind the stuck request of A
        assert srv.wait(srv.submit(B, "project", "fp32"), 60000) == 0   # B is still served
        assert srv.cancel(t3) == 0
        assert srv.wait(t3, 1000) == ERR_CANCELLED
        assert srv.cancel(t1) == ERR_STATE             # already started: not cancellable
        assert srv.cancel(987654) == ERR_STATE
        srv.fault_hold(A, False)
        assert srv.wait(t1, 60000) == 0
        _, ca = srv.read(A, psi=False)
        psi_after, _ = srv.read(A, coeff=False)
        # the cancelled expansion never ran: psi of A is unchanged
        assert bool((psi_after == psia.cpu()).all())
        # a held request does not keep the server from shutting down
        srv.fault_hold(B, True)
        srv.submit(B, "project", "fp32")
        closer = threading.Thread(target=srv.close)
        closer.start()
        closer.join(60)
        assert not closer.is_alive(), "server shutdown waited on a held request"
    direct = api.project(psia, pa, sa, nua, 32, 0.2, True, prec="fp32")
    import torch
    assert torch.equal(direct.cpu(), ca)


def test_status_names():
    from paper_1905_00480_gb300 import _native as N
    assert N.STATUS_NAMES[ERR_CANCELLED] == "SHO_ERR_CANCELLED"
    assert N.lib().sho_strerror(ERR_CANCELLED) not in (None, b"unknown status")
