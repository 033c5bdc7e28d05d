"""FP64-accurate expansion with the x-pass on the tensor cores by exact digit slicing (GPU).

First the MMA schedule in isolation: six TF32 digit slices of each operand (integers of at most 128 times
2^(-8 i)), every digit pair with i + j <= 8 accumulated into its level accumulator; the leading three
levels must equal the exact sums bit for bit, the merged fourth to FP32 rounding.  Then the expansion
built on it against the oracle at the FP64 bar, and against the float-float CUDA-core kernel, on the
geometries that stress the tile bookkeeping: partial 128-band tiles, two band tiles, clipped cubes, cubes
starting inside a tile on a periodic grid, numax 0 and 7, many atoms per tile, a wide dynamic range of
coefficients, and the bounded waits running out under an injected staging stop."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu

ERR_TIMEOUT = -8
SHORT_WAIT = 200_000      # SM clock cycles, ~0.1 ms: far below the ~2 s default


def _digits(rng, shape, maxabs=128):
    """Six digit slices: slice i - 1 holds integers in [-maxabs, maxabs] times 2^(-8 i)."""
    d = rng.integers(-maxabs, maxabs + 1, size=(6,) + shape).astype(np.float64)
    return d * (2.0 ** (-8.0 * np.arange(1, 7)))[:, None, None]


@pytest.mark.parametrize("maxabs", [128, 5])
def test_ozaki_schedule_selftest(maxabs):
    require_gpu()
    from paper_1905_00480_gb300 import _native as N
    rng = np.random.default_rng(70 + maxabs)
    A = _digits(rng, (128, 8), maxabs)
    B = _digits(rng, (32, 8), maxabs)
    ref = np.zeros((4, 128, 32))
    for i in range(1, 7):
        for j in range(1, 7):
            if i + j <= 8:
                ref[min(i + j, 5) - 2] += A[i - 1] @ B[j - 1].T   # exact in FP64 (integers times 2^-8L)
    Af, Bf = A.astype(np.float32), B.astype(np.float32)
    assert np.array_equal(Af.astype(np.float64), A) and np.array_equal(Bf.astype(np.float64), B)
    D = np.zeros((4, 128, 32), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    st = N.lib().sho_selftest_ozaki(Af.ctypes.data_as(fp), Bf.ctypes.data_as(fp), D.ctypes.data_as(fp))
    assert st == 0, N.STATUS_NAMES.get(st, st)
    for g in range(3):   # levels 2, 3, 4: exact integer sums
        assert np.array_equal(D[g].astype(np.float64), ref[g]), (g, np.argwhere(D[g] != ref[g])[:5])
    scale = np.abs(ref[3]).max() + 1e-300
    assert np.abs(D[3] - ref[3]).max() <= 1e-6 * scale


def _t(x):
    import torch
    return torch.from_numpy(np.ascontiguousarray(x)).cuda()


def _expand_both(grid, h, periodic, pos, sig, psi, c, numax, cube):
    """FF64 expansion with the tensor-core x-pass (chosen) and with the float-float kernel; the default
    engine is the tensor-core one when the bands fill its 128-band tiles at least three quarters, the
    float-float one otherwise, bit for bit."""
    from paper_1905_00480_gb300 import api
    outs = {}
    for kernel in ("tcgen05", "auto", "mma_sync"):
        hd = api.Handle(0)
        hd.set_expand_kernel(kernel)
        out = _t(psi)
        api.add(out, _t(c), pos, sig, numax, cube, h, periodic, prec="ff64", handle=hd)
        hd.sync()
        outs[kernel] = out.cpu().numpy()
        hd.close()
    nb = psi.shape[3]
    full = 4 * nb >= 3 * 128 * ((nb + 127) // 128)
    assert np.array_equal(outs["auto"], outs["tcgen05" if full else "mma_sync"])
    return outs["tcgen05"], outs["mma_sync"]


@pytest.mark.parametrize("grid,periodic,numax,cube,nbands,natoms", [
    ((56, 40, 36), True, 5, 16, 64, 7),     # one partial band tile (64 of 128)
    ((44, 38, 30), False, 3, 16, 130, 5),   # clipped cubes; band tiles of 128 + 2
    ((64, 48, 40), True, 7, 32, 32, 4),     # numax 7 (8 states), cube 32 on the narrowest grid allowed
    ((48, 48, 48), True, 0, 16, 8, 6),      # numax 0
    ((48, 34, 32), True, 5, 16, 16, 40),    # many atoms per tile: the exact levels under load
])
def test_ozaki_expansion_matches_oracle(grid, periodic, numax, cube, nbands, natoms):
    require_gpu()
    rng = np.random.default_rng(7100 + 10 * numax + natoms)
    h = 0.2
    pos, sig = workloads.random_atoms(rng, natoms, tuple(n * h for n in grid), periodic,
                                      min_sep=0.3 if natoms > 10 else 1.0)
    if not periodic:
        pos[0] = [0.1 * h, 0.5 * grid[1] * h, 0.5 * grid[2] * h]
        pos[1] = [(grid[0] - 0.3) * h, 0.3 * grid[1] * h, (grid[2] - 0.6) * h]
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((natoms, oracle.nstates(numax), nbands))
    got, ff = _expand_both(grid, h, periodic, pos, sig, psi, c, numax, cube)
    ref = oracle.add(grid, h, periodic, psi, pos, sig, numax, cube, c)
    assert rel_norm(got - psi, ref - psi) <= TOL_FP64
    assert rel_max(got - psi, ref - psi) <= TOL_FP64
    assert rel_norm(got - psi, ff - psi) <= TOL_FP64
    assert not np.array_equal(got, ff)   # the two kernels round differently: the tensor-core path ran


def test_ozaki_expansion_wide_dynamic_range_and_determinism():
    """Per-atom coefficient scales from 1e-12 to 1e12 expanded into a zero grid: each point's frame
    follows the largest contribution; norm-wise FP64 accuracy, and bit-identical repeated runs."""
    require_gpu()
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(7200)
    grid, h, periodic, numax, cube, nbands = (64, 40, 36), 0.2, True, 5, 32, 24
    pos, sig = workloads.random_atoms(rng, 6, tuple(n * h for n in grid), periodic, min_sep=1.0)
    c = rng.standard_normal((6, oracle.nstates(numax), nbands)) * 10.0 ** rng.uniform(-12, 12, size=(6, 1, 1))
    zero = np.zeros((grid[2], grid[1], grid[0], nbands))
    hd = api.Handle(0)
    hd.set_expand_kernel("tcgen05")
    runs = []
    for _ in range(2):
        out = _t(zero)
        api.add(out, _t(c), pos, sig, numax, cube, h, periodic, prec="ff64", handle=hd)
        runs.append(out.cpu().numpy())
    hd.close()
    assert np.array_equal(runs[0], runs[1])
    ref = oracle.add(grid, h, periodic, zero, pos, sig, numax, cube, c)
    assert rel_norm(runs[0], ref) <= TOL_FP64
    assert rel_max(runs[0], ref) <= TOL_FP64


def test_ozaki_bounded_wait_runs_out_and_next_call_is_clean():
    """The z-pass slices of only the first atom of each tile are staged (sho_fault_stop_rows) under a
    short wait limit: the wait for the second atom's slice runs out, the kernel drains its copies and
    MMAs and returns, and sho_sync reports SHO_ERR_TIMEOUT; the next normal call is correct."""
    require_gpu()
    from paper_1905_00480_gb300 import _native as N
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(7300)
    grid, h, periodic, numax, cube, nbands = (56, 40, 36), 0.2, True, 5, 16, 32
    pos, sig = workloads.random_atoms(rng, 12, tuple(n * h for n in grid), periodic, min_sep=1.0)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands))
    c = rng.standard_normal((12, oracle.nstates(numax), nbands))
    hd = api.Handle(0)
    hd.set_expand_kernel("tcgen05")
    L = N.lib()
    assert L.sho_fault_wait_limit(hd.ptr, SHORT_WAIT) == 0
    assert L.sho_fault_stop_rows(hd.ptr, 1) == 0
    out = _t(psi)
    api.add(out, _t(c), pos, sig, numax, cube, h, periodic, prec="ff64", handle=hd)
    assert L.sho_sync(hd.ptr) == ERR_TIMEOUT
    assert L.sho_sync(hd.ptr) == 0
    assert L.sho_fault_wait_limit(hd.ptr, 0) == 0
    assert L.sho_fault_stop_rows(hd.ptr, -1) == 0
    out = _t(psi)
    api.add(out, _t(c), pos, sig, numax, cube, h, periodic, prec="ff64", handle=hd)
    assert L.sho_sync(hd.ptr) == 0
    ref = oracle.add(grid, h, periodic, psi, pos, sig, numax, cube, c)
    assert rel_norm(out.cpu().numpy() - psi, ref - psi) <= TOL_FP64
    hd.close()
