"""Fifth-generation tensor-core path (tcgen05 MMA, tensor memory) of the TF32 / BF16 / 3xTF32 /
split-FP16 expansion (GPU).

First the operand layouts in isolation: one M=128, N=32 MMA on integer-valued operands, whose products
and sums are exact in FP32, must equal numpy's matrix product bit for bit.  Then the expansion kernel
built on it against the oracle (and against the warp-level MMA kernel) on the geometries that stress the
tile bookkeeping: ragged band counts (partial 128-band tiles), wrapped and clipped cubes, cubes wider
than a tile, several atoms per tile."""
import ctypes

import numpy as np
import pytest

import oracle
import workloads
from helpers import rel_norm, require_gpu
from test_parity_tc import TOL

pytestmark = pytest.mark.gpu


@pytest.mark.parametrize("bf16", [0, 1])
def test_umma_layout_selftest(bf16):
    require_gpu()
    from paper_1905_00480_gb300 import _native as N
    K = 16 if bf16 else 8
    rng = np.random.default_rng(40 + bf16)
    A = rng.integers(-8, 9, size=(128, K)).astype(np.float32)
    B = rng.integers(-8, 9, size=(32, K)).astype(np.float32)
    D = np.zeros((128, 32), dtype=np.float32)
    fp = ctypes.POINTER(ctypes.c_float)
    st = N.lib().sho_selftest_umma(bf16, A.ctypes.data_as(fp), B.ctypes.data_as(fp), D.ctypes.data_as(fp))
    assert st == 0, N.STATUS_NAMES.get(st, st)
    assert np.array_equal(D, A @ B.T), np.argwhere(D != A @ B.T)[:10]


@pytest.mark.parametrize("mode", ["tf32", "bf16", "3xtf32", "split_fp16"])
@pytest.mark.parametrize("grid,periodic,numax,cube,nbands", [
    ((40, 36, 44), True, 7, 32, 200),    # 128 + 72 bands: a partial band tile
    ((34, 40, 36), True, 5, 32, 64),     # periodic grid barely wider than the cube: wrapped tiles
    ((40, 36, 44), False, 3, 16, 36),    # clipped cubes, 36 bands
    ((64, 52, 56), False, 6, 48, 128),   # cubes wider than a tile
])
def test_umma_expansion_matches_oracle(mode, grid, periodic, numax, cube, nbands):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(4100 + numax + cube)
    h = 0.2
    pos, sig = workloads.random_atoms(rng, 7, tuple(n * h for n in grid), periodic, min_sep=1.0)
    if not periodic:
        pos[0] = [0.1 * h, 0.5 * grid[1] * h, 0.5 * grid[2] * h]
        pos[1] = [(grid[0] - 0.3) * h, 0.3 * grid[1] * h, 0.6 * grid[2] * h]
    c = rng.standard_normal((7, oracle.nstates(numax), nbands)).astype(np.float32)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)).astype(np.float32)
    outs = {}
    for kernel in ("tcgen05", "mma_sync"):
        hd = api.Handle(0)
        hd.set_expand_kernel(kernel)
        out = torch.from_numpy(psi).cuda()
        api.add(out, torch.from_numpy(c).cuda(), pos, sig, numax, cube, h, periodic, prec=mode, handle=hd)
        hd.sync()
        outs[kernel] = out.double().cpu().numpy() - psi
        hd.close()
    ref = oracle.add(grid, h, periodic, np.zeros(psi.shape), pos, sig, numax, cube, c.astype(np.float64))
    assert rel_norm(outs["tcgen05"], ref) <= TOL[mode]
    # the same products in the same atom order: the two engines agree far inside the form's bound
    assert rel_norm(outs["tcgen05"], outs["mma_sync"]) <= TOL[mode] / 10


def test_umma_bf16_storage_and_c160_sample():
    """BF16-stored psi through the tensor-memory tile, and the 160^3 precision workload on sampled points."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    w = workloads.WORKLOADS["c160"]
    pos, sig = workloads.atoms(w)
    N = oracle.nstates(w.numax)
    c = torch.from_numpy(workloads.coeff_host(w, N)).to("cuda", torch.float32)
    out = torch.zeros((w.grid[2], w.grid[1], w.grid[0], w.nbands), dtype=torch.bfloat16, device="cuda")
    hd = api.Handle(0)
    hd.set_expand_kernel("tcgen05")
    api.add(out, c, pos, sig, w.numax, w.cube, w.h, w.periodic, prec="tf32", handle=hd)
    hd.sync()
    rng = np.random.default_rng(4200)
    pts = np.sort(rng.choice(w.grid[0] * w.grid[1] * w.grid[2], size=300, replace=False))
    got = out.reshape(-1, w.nbands)[torch.from_numpy(pts).cuda()][:, :32].double().cpu().numpy()
    ref = oracle.expand_points(w.grid, w.h, w.periodic, pos, sig, w.numax, w.cube,
                               c[:, :, :32].double().cpu().numpy(), pts)
    assert rel_norm(got, ref) <= TOL["tf32"] + 2.0 ** -8
    hd.close()
