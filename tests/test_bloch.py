"""Bloch (complex) projection and expansion on the GPU against the oracle (FP64 and FP64-accurate forms,
1e-12; FP32 form on complex64 data against the oracle run on the same rounded input, the FP32 bound)."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, TOL_FP64, assert_coeff_close, rel_norm, require_gpu

pytestmark = pytest.mark.gpu


def _case(seed, grid, h, natoms, nbands):
    rng = np.random.default_rng(seed)
    L = np.array(grid) * h
    pos, sig = workloads.random_atoms(rng, natoms, tuple(L), True, min_sep=1.0)
    pos[0] = [0.3 * h + 0.01, L[1] - 0.4 * h, 0.6 * h]  # a cube that wraps on every axis
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)) + 1j * rng.standard_normal(
        (grid[2], grid[1], grid[0], nbands))
    return rng, pos, sig, psi


@pytest.mark.parametrize("prec", ["fp64", "ff64"])
@pytest.mark.parametrize("numax,nbands", [(3, 5), (5, 40), (7, 33)])
def test_bloch_project_and_add(numax, nbands, prec):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, cube = (40, 36, 34), 0.2, 32
    rng, pos, sig, psi = _case(910 + numax, grid, h, 5, nbands)
    k = np.array([0.9, -0.35, 1.7])
    psi_d = torch.from_numpy(psi).cuda()
    got = api.project_bloch(psi_d, k, pos, sig, numax, cube, h, prec=prec).cpu().numpy()
    ref = oracle.project_bloch(grid, h, k, psi, pos, sig, numax, cube)
    assert_coeff_close(got.view(np.float64), ref.view(np.float64), TOL_FP64)
    coef = rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)
    out = psi_d.clone()
    api.add_bloch(out, torch.from_numpy(coef).cuda(), k, pos, sig, numax, cube, h, prec=prec)
    ref2 = oracle.add_bloch(grid, h, k, psi, pos, sig, numax, cube, coef)
    assert rel_norm((out.cpu().numpy() - psi).view(np.float64), (ref2 - psi).view(np.float64)) <= TOL_FP64


@pytest.mark.parametrize("numax,nbands,k", [(3, 6, (0.0, 0.0, 0.0)), (5, 40, (0.9, -0.35, 1.7)),
                                            (7, 34, (-2.2, 1.3, 0.6))])
def test_bloch_fp32_project_and_add(numax, nbands, k):
    """FP32 form on complex64 data (the real FP32 CUDA-core kernels over the (re, im) pairs, the phases
    applied in FP32): 2 nbands real bands over full and ragged 32-band tiles, cubes that wrap on every
    axis, k = 0 included."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, cube = (40, 36, 34), 0.2, 32
    rng, pos, sig, psi = _case(950 + numax, grid, h, 5, nbands)
    psi_d = torch.from_numpy(psi.astype(np.complex64)).cuda()
    psi_r = psi_d.cpu().numpy().astype(np.complex128)   # the rounded input the kernels see
    k = np.array(k)
    got = api.project_bloch(psi_d, k, pos, sig, numax, cube, h, prec="fp32")
    assert got.dtype == torch.complex64
    ref = oracle.project_bloch(grid, h, k, psi_r, pos, sig, numax, cube)
    assert_coeff_close(got.cpu().numpy().astype(np.complex128).view(np.float64), ref.view(np.float64), TOL_FP32)
    coef_d = torch.from_numpy((rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)).astype(
        np.complex64)).cuda()
    out = psi_d.clone()
    api.add_bloch(out, coef_d, k, pos, sig, numax, cube, h, prec="fp32")
    ref2 = oracle.add_bloch(grid, h, k, psi_r, pos, sig, numax, cube, coef_d.cpu().numpy().astype(np.complex128))
    d = out.cpu().numpy().astype(np.complex128) - psi_r
    assert rel_norm(d.view(np.float64), (ref2 - psi_r).view(np.float64)) <= TOL_FP32


def test_bloch_fp32_adjoint():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, numax, cube = (40, 36, 34), 0.2, 6, 32
    rng, pos, sig, psi = _case(955, grid, h, 4, 8)
    psi_d = torch.from_numpy(psi.astype(np.complex64)).cuda()
    k = [1.1, 0.4, -0.8]
    c = api.project_bloch(psi_d, k, pos, sig, numax, cube, h, prec="fp32")
    coef = torch.from_numpy((rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).astype(
        np.complex64)).cuda()
    ec = api.add_bloch(torch.zeros_like(psi_d), coef, k, pos, sig, numax, cube, h, prec="fp32")
    lhs = torch.vdot(c.flatten().cdouble(), coef.flatten().cdouble()).item()
    rhs = h ** 3 * torch.vdot(psi_d.flatten().cdouble(), ec.flatten().cdouble()).item()
    assert abs(lhs - rhs) <= 1e-5 * abs(lhs)


@pytest.mark.parametrize("prec", ["ff64", "fp32"])
def test_bloch_cubes_across_every_cell_face(prec):
    """Atoms on both sides of every face and in the corners, so that cube rows cross the boundary at
    their start and at their end along each axis, and tile segments meet both runs; a grid wider than
    the FP64 expansion's row limit."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, cube, numax, nbands = (456, 40, 36), 0.2, 16, 4, 6
    cdt, tol = (np.complex128, TOL_FP64) if prec == "ff64" else (np.complex64, TOL_FP32)
    L = np.array(grid) * h
    rng = np.random.default_rng(941)
    pos = np.array([[0.05 * h, 0.3 * h, 0.2 * h], [L[0] - 0.3 * h, L[1] - 0.1 * h, L[2] - 0.45 * h],
                    [L[0] / 2, 0.4 * h, L[2] - 0.2 * h], [0.6 * h, L[1] / 2, L[2] / 2],
                    [L[0] - 2.3 * h, 2.7 * h, 1.1 * h]])
    sig = np.full(len(pos), 0.75)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)) + 1j * rng.standard_normal(
        (grid[2], grid[1], grid[0], nbands))
    k = np.array([-1.3, 0.8, 2.1])
    psi = psi.astype(cdt).astype(np.complex128)
    psi_d = torch.from_numpy(psi.astype(cdt)).cuda()
    got = api.project_bloch(psi_d, k, pos, sig, numax, cube, h, prec=prec).cpu().numpy().astype(np.complex128)
    ref = oracle.project_bloch(grid, h, k, psi, pos, sig, numax, cube)
    assert_coeff_close(got.view(np.float64), ref.view(np.float64), tol)
    coef = (rng.standard_normal(ref.shape) + 1j * rng.standard_normal(ref.shape)).astype(cdt).astype(np.complex128)
    out = torch.zeros_like(psi_d)
    api.add_bloch(out, torch.from_numpy(coef.astype(cdt)).cuda(), k, pos, sig, numax, cube, h, prec=prec)
    ref2 = oracle.add_bloch(grid, h, k, np.zeros_like(psi), pos, sig, numax, cube, coef)
    got2 = out.cpu().numpy().astype(np.complex128)
    assert rel_norm(got2.view(np.float64), ref2.view(np.float64)) <= tol


def test_bloch_ff64_zero_k_is_the_real_form_on_each_part():
    """k = 0: every phase is 1 and the FP64-accurate Bloch kernels are the real ones over the (re, im)
    pairs, so each part matches the real FP64-accurate projection and expansion bit for bit."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, numax, cube = (40, 36, 34), 0.2, 5, 32
    rng, pos, sig, psi = _case(925, grid, h, 4, 12)
    psi_d = torch.from_numpy(psi).cuda()
    c0 = api.project_bloch(psi_d, [0, 0, 0], pos, sig, numax, cube, h, prec="ff64")
    hf = api.Handle(0)
    hf.set_project_kernel("mma_sync")  # the float-float projection, the engine of the Bloch form
    cr = api.project(psi_d.real.contiguous(), pos, sig, numax, cube, h, True, prec="ff64", handle=hf)
    ci = api.project(psi_d.imag.contiguous(), pos, sig, numax, cube, h, True, prec="ff64", handle=hf)
    hf.close()
    assert torch.equal(c0.real.contiguous(), cr) and torch.equal(c0.imag.contiguous(), ci)
    coef = torch.from_numpy(rng.standard_normal(c0.shape) + 1j * rng.standard_normal(c0.shape)).cuda()
    out = psi_d.clone()
    api.add_bloch(out, coef, [0, 0, 0], pos, sig, numax, cube, h, prec="ff64")
    re, im = psi_d.real.contiguous(), psi_d.imag.contiguous()
    hd = api.Handle(0)
    hd.set_expand_kernel("mma_sync")  # the float-float block gather, the engine of the Bloch form
    api.add(re, coef.real.contiguous(), pos, sig, numax, cube, h, True, prec="ff64", handle=hd)
    api.add(im, coef.imag.contiguous(), pos, sig, numax, cube, h, True, prec="ff64", handle=hd)
    hd.close()
    assert torch.equal(out.real.contiguous(), re) and torch.equal(out.imag.contiguous(), im)


def test_bloch_ff64_adjoint_and_fp64_agreement():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, numax, cube = (40, 36, 34), 0.2, 6, 32
    rng, pos, sig, psi = _case(935, grid, h, 4, 7)
    psi_d = torch.from_numpy(psi).cuda()
    k = [1.1, 0.4, -0.8]
    c = api.project_bloch(psi_d, k, pos, sig, numax, cube, h, prec="ff64")
    c64 = api.project_bloch(psi_d, k, pos, sig, numax, cube, h, prec="fp64")
    assert rel_norm(torch.view_as_real(c).cpu().numpy(), torch.view_as_real(c64).cpu().numpy()) <= TOL_FP64
    coef = torch.from_numpy(rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).cuda()
    ec = api.add_bloch(torch.zeros_like(psi_d), coef, k, pos, sig, numax, cube, h, prec="ff64")
    lhs = torch.vdot(c.flatten(), coef.flatten()).item()
    rhs = h ** 3 * torch.vdot(psi_d.flatten(), ec.flatten()).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_bloch_rejects_other_precisions():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api, ShoError
    pos = np.array([[2.0, 2.0, 2.0]])
    psi = torch.zeros((16, 16, 16, 2), dtype=torch.complex128, device="cuda")
    for prec in ("tf32", "bf16", "3xtf32"):
        with pytest.raises(ShoError):
            api.project_bloch(psi, [0.1, 0, 0], pos, [1.0], 1, 16, 0.25, prec=prec)
    with pytest.raises(ValueError):   # FP32 form: complex64 data
        api.project_bloch(psi, [0.1, 0, 0], pos, [1.0], 1, 16, 0.25, prec="fp32")
    odd = torch.zeros((16, 16, 16, 3), dtype=torch.complex64, device="cuda")
    with pytest.raises(ShoError):     # FP32 form: 2 nbands real bands in 16-byte rows
        api.project_bloch(odd, [0.1, 0, 0], pos, [1.0], 1, 16, 0.25, prec="fp32")
    flat = torch.zeros(16 * 16 * 16 * 2 + 1, dtype=torch.complex64, device="cuda")
    shifted = flat[1:].view(16, 16, 16, 2)   # contiguous, 8 bytes past a 16-byte boundary
    assert shifted.data_ptr() % 16 == 8
    with pytest.raises(ShoError):
        api.project_bloch(shifted, [0.1, 0, 0], pos, [1.0], 1, 16, 0.25, prec="fp32")
    c = torch.zeros((1, oracle.nstates(1), 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(ShoError):
        api.add_bloch(shifted, c, [0.1, 0, 0], pos, [1.0], 1, 16, 0.25, prec="fp32")
    ok = torch.zeros((16, 16, 16, 2), dtype=torch.complex64, device="cuda")
    with pytest.raises(ShoError):     # numax above 7
        api.project_bloch(ok, [0.1, 0, 0], pos, [1.0], 8, 16, 0.25, prec="fp32")


def test_bloch_zero_k_matches_real_path_and_adjoint():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, numax, cube = (40, 36, 34), 0.2, 5, 32
    rng, pos, sig, psi = _case(920, grid, h, 4, 16)
    psi_d = torch.from_numpy(psi).cuda()
    c0 = api.project_bloch(psi_d, [0, 0, 0], pos, sig, numax, cube, h)
    cr = api.project(psi_d.real.contiguous(), pos, sig, numax, cube, h, True, prec="fp64")
    ci = api.project(psi_d.imag.contiguous(), pos, sig, numax, cube, h, True, prec="fp64")
    assert rel_norm(c0.real.cpu().numpy(), cr.cpu().numpy()) <= TOL_FP64
    assert rel_norm(c0.imag.cpu().numpy(), ci.cpu().numpy()) <= TOL_FP64
    # adjoint identity on the GPU path, k != 0
    k = [1.1, 0.4, -0.8]
    c = api.project_bloch(psi_d, k, pos, sig, numax, cube, h)
    coef = torch.from_numpy(rng.standard_normal(c.shape) + 1j * rng.standard_normal(c.shape)).cuda()
    ec = api.add_bloch(torch.zeros_like(psi_d), coef, k, pos, sig, numax, cube, h)
    lhs = torch.vdot(c.flatten(), coef.flatten()).item()
    rhs = h ** 3 * torch.vdot(psi_d.flatten(), ec.flatten()).item()
    assert abs(lhs - rhs) <= 1e-12 * abs(lhs)


def test_bloch_rejects_open_grid():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api, ShoError
    from paper_1905_00480_gb300 import _native as N
    import ctypes
    psi = torch.zeros((16, 16, 16, 2), dtype=torch.complex128, device="cuda")
    out = torch.zeros((1, 4, 2), dtype=torch.complex128, device="cuda")
    g = N.sho_grid()
    g.n[0] = g.n[1] = g.n[2] = 16
    g.h, g.periodic = 0.25, 0
    k = np.zeros(3)
    pos = np.array([[2.0, 2.0, 2.0]])
    sig = np.array([1.0])
    st = N.lib().sho_project_bloch(api.default_handle(0).ptr, ctypes.byref(g), k.ctypes.data_as(N._DP),
                                   ctypes.c_void_p(psi.data_ptr()), 2, 1, pos.ctypes.data_as(N._DP),
                                   sig.ctypes.data_as(N._DP), 1, 16, N.PRECS["fp64"], ctypes.c_void_p(out.data_ptr()),
                                   None)
    assert st != 0


def test_bloch_ff64_tensor_core_expansion():
    """On a grid at least cube + 32 points wide the FF64 Bloch expansion can take the tensor-core x-pass
    (T1 turned by its tile's phase before the digit slicing): against the oracle with cubes that wrap on
    every axis, and against the float-float block gather (close, not bit for bit); with 20 complex bands
    (40 real, a third of a 128-band tile) the automatic choice is the block gather."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    grid, h, cube, numax, nbands = (72, 40, 36), 0.2, 32, 5, 20
    rng, pos, sig, psi = _case(945, grid, h, 5, nbands)
    k = np.array([0.7, -1.2, 0.45])
    coef = rng.standard_normal((len(pos), oracle.nstates(numax), nbands)) + 1j * rng.standard_normal(
        (len(pos), oracle.nstates(numax), nbands))
    outs = {}
    for engine in ("tcgen05", "mma_sync", "auto"):
        hd = api.Handle(0)
        hd.set_expand_kernel(engine)
        out = torch.zeros((grid[2], grid[1], grid[0], nbands), dtype=torch.complex128, device="cuda")
        api.add_bloch(out, torch.from_numpy(coef).cuda(), k, pos, sig, numax, cube, h, handle=hd, prec="ff64")
        hd.sync()
        outs[engine] = out.cpu().numpy()
        hd.close()
    ref = oracle.add_bloch(grid, h, k, np.zeros_like(psi), pos, sig, numax, cube, coef)
    for engine, got in outs.items():
        assert rel_norm(got.view(np.float64), ref.view(np.float64)) <= TOL_FP64, engine
    assert not np.array_equal(outs["tcgen05"], outs["mma_sync"])  # the tensor-core path ran
    assert np.array_equal(outs["auto"], outs["mma_sync"])
