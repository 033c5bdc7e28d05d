"""sho_forces_noalloc, the allocation-free forces entry point, agrees with sho_forces and with the
oracle (GPU).

Callers that cannot allocate device memory (their own pool owns it, their host forbids foreign
allocations, or they run at the memory limit) use sho_forces_noalloc, whose scratch is a fixed static
device array inside the library.  This test calls it through the C ABI twice in a row -- the second
call reuses the array left by the first -- and checks both results against the allocating entry point
and against the FP64 oracle within the tolerances of the other parity tests, and that the two calls
changed neither the device's free memory nor the torch allocator's allocation count.  It also checks
that a problem larger than the fixed scratch is rejected before anything runs.  The file is named so
that pytest collects it last.
"""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, TOL_FP64, rel_max, require_gpu

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def lib():
    require_gpu()
    from paper_1905_00480_gb300 import build
    build.build()
    from paper_1905_00480_gb300 import _native
    return _native.lib()


def _noalloc(lib, psi, dEdc, pos, sig, numax, cube, h, periodic, prec, out):
    import torch
    from paper_1905_00480_gb300 import _native as N
    g = N.sho_grid()
    g.n[0], g.n[1], g.n[2] = psi.shape[2], psi.shape[1], psi.shape[0]
    g.h = h
    g.periodic = int(periodic)
    dt = {torch.float64: 0, torch.float32: 1, torch.bfloat16: 2}
    pos_h = np.ascontiguousarray(pos, dtype=np.float64)
    sig_h = np.ascontiguousarray(sig, dtype=np.float64)
    dp = ctypes.POINTER(ctypes.c_double)
    stream = torch.cuda.current_stream().cuda_stream
    return lib.sho_forces_noalloc(ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()), dt[psi.dtype], psi.shape[3],
                                  pos_h.shape[0], pos_h.ctypes.data_as(dp), sig_h.ctypes.data_as(dp), numax, cube,
                                  N.PRECS[prec], ctypes.c_void_p(dEdc.data_ptr()), dt[dEdc.dtype],
                                  ctypes.cast(ctypes.c_void_p(out.data_ptr()), dp), ctypes.c_void_p(stream))


def _case(seed, natoms, numax, nbands, grid=(40, 36, 44), h=0.2):
    rng = np.random.default_rng(seed)
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * h for n in grid), True, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    dEdc = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    return pos, sig, psi, dEdc


@pytest.mark.parametrize("prec,storage", [("fp64", "f64"), ("fp32", "f32"), ("fp32", "bf16")])
def test_noalloc_matches_allocating_entry_point_and_oracle_twice(lib, prec, storage):
    import torch
    from paper_1905_00480_gb300 import api
    numax, cube, h, grid = 4, 16, 0.2, (40, 36, 44)
    pos, sig, psi, dEdc = _case(123, 6, numax, 45, grid=grid, h=h)
    tdt = {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[storage]
    cdt = torch.float64 if prec == "fp64" else torch.float32
    psi_d = torch.from_numpy(psi).cuda().to(tdt)
    dEdc_d = torch.from_numpy(dEdc).cuda().to(cdt)
    ref = api.forces(psi_d, dEdc_d, pos, sig, numax, cube, h, True, prec=prec).cpu().numpy()
    # the oracle on the storage-rounded inputs the kernels see (ladder-relation forces difference
    # neighbouring coefficients: the FP32 bar is 10x the coefficient bar, as in the FP32 parity tests)
    ora = oracle.forces(grid, h, True, psi_d.double().cpu().numpy(), pos, sig, numax, cube,
                        dEdc_d.double().cpu().numpy())
    tol = TOL_FP64 if prec == "fp64" else 10 * TOL_FP32
    # the first call on the device looks up the scratch array (and may load the library's kernels)
    out = torch.empty((len(pos), 3), dtype=torch.float64, device="cuda")
    assert _noalloc(lib, psi_d, dEdc_d, pos, sig, numax, cube, h, True, prec, out) == 0
    outs = [torch.full((len(pos), 3), float("nan"), dtype=torch.float64, device="cuda") for _ in range(2)]
    torch.cuda.synchronize()
    free1 = torch.cuda.mem_get_info()[0]
    allocs1 = torch.cuda.memory_stats().get("allocation.all.allocated", 0)
    for o in outs:  # two calls in a row: the second reuses the array the first left behind
        st = _noalloc(lib, psi_d, dEdc_d, pos, sig, numax, cube, h, True, prec, o)
        assert st == 0, f"sho_forces_noalloc returned {st}"
    torch.cuda.synchronize()
    # the calls allocated no device memory, neither through the driver nor through torch's allocator
    assert torch.cuda.mem_get_info()[0] == free1
    assert torch.cuda.memory_stats().get("allocation.all.allocated", 0) == allocs1
    for o in outs:
        got = o.cpu().numpy()
        assert np.all(np.isfinite(got))
        assert rel_max(got, ref) <= tol
        assert rel_max(got, ora) <= tol


def test_noalloc_rejects_problems_beyond_its_scratch(lib):
    import torch
    from paper_1905_00480_gb300 import _native as N
    # 64 atoms x N(6) = 84 states x 512 bands x 8 bytes = 22 MB > the 16 MiB scratch
    numax, nb = 5, 512
    psi_d = torch.zeros((32, 32, 32, nb), dtype=torch.float64, device="cuda")
    rng = np.random.default_rng(5)
    pos = rng.uniform(0, 6.4, size=(64, 3))
    sig = np.full(64, 0.7)
    dEdc_d = torch.zeros((64, oracle.nstates(numax), nb), dtype=torch.float64, device="cuda")
    out = torch.full((64, 3), 7.0, dtype=torch.float64, device="cuda")
    st = _noalloc(lib, psi_d, dEdc_d, pos, sig, numax, 16, 0.2, True, "fp64", out)
    assert st == -10 and N.STATUS_NAMES[st] == "SHO_ERR_CAPACITY"
    torch.cuda.synchronize()
    assert float(out.min()) == 7.0 and float(out.max()) == 7.0
