"""Plane-sweep projection of the FP32-class forms (FP32 or BF16 psi, numax <= 7) against the FP64 oracle
run on the storage-rounded psi (GPU), and the FP32-class expansion on the same geometries.

The plane sweep assigns every (atom, plane) row segment to a register slot on the host; these cases
drive its corners: more overlapping atoms per row than slots (several sweeps of one plane), wrapped
cubes on grids barely larger than the cube (both halves of a wrapped atom in one warp), atoms far
outside a non-periodic box, every numax, and the fallback to the per-atom kernels when a row does not
fit one TMA box."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, assert_coeff_close, rel_norm, require_gpu
from test_parity_tc import TOL

pytestmark = pytest.mark.gpu


def _project(grid, h, periodic, pos, sig, numax, cube, nbands, prec, seed, storage="f32"):
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)).astype(np.float32)
    psi_d = torch.from_numpy(psi).cuda().to(torch.bfloat16 if storage == "bf16" else torch.float32)
    assert api.project_path(psi_d, numax, cube, h, periodic, prec=prec) == "plane"
    got = api.project(psi_d, pos, sig, numax, cube, h, periodic, prec=prec).double().cpu().numpy()
    ref = oracle.project(grid, h, periodic, psi_d.double().cpu().numpy(), pos, sig, numax, cube)
    return got, ref


def _tol(prec):
    return TOL_FP32 if prec == "fp32" else TOL[prec]


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "3xtf32", "bf16", "split_fp16"])
def test_dense_atoms_need_several_sweeps(prec, storage):
    """120 atoms in a periodic 48^3 box with cube 32: about 53 cubes meet each grid row, more than the
    33 register slots of one sweep, so planes are swept more than once."""
    require_gpu()
    rng = np.random.default_rng(601)
    grid, h, numax, cube = (48, 48, 48), 0.2, 3, 32
    pos, sig = workloads.random_atoms(rng, 120, tuple(n * h for n in grid), True, min_sep=0.6)
    got, ref = _project(grid, h, True, pos, sig, numax, cube, 8, prec, 602, storage)
    assert_coeff_close(got, ref, _tol(prec))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
@pytest.mark.parametrize("prec", ["fp32", "tf32", "bf16"])
def test_wrapped_cubes_on_small_grid(prec, storage):
    """Periodic grid only 2-4 points longer than the cube in y: most cubes wrap, and the two halves of a
    wrapped atom are summed in one warp."""
    require_gpu()
    rng = np.random.default_rng(603)
    grid, h, numax, cube = (36, 34, 40), 0.2, 5, 32
    pos, sig = workloads.random_atoms(rng, 7, tuple(n * h for n in grid), True, min_sep=1.0)
    got, ref = _project(grid, h, True, pos, sig, numax, cube, 40 if storage == "bf16" else 36, prec, 604, storage)
    assert_coeff_close(got, ref, _tol(prec))


@pytest.mark.parametrize("storage", ["f32", "bf16"])
def test_atoms_outside_open_box(storage):
    """Not periodic: cubes clipped on every side, and one atom whose cube misses the grid in y entirely
    (its coefficients are exactly zero)."""
    require_gpu()
    grid, h, numax, cube = (40, 40, 40), 0.25, 4, 32
    L = 40 * h
    pos = np.array([[-2.0, 3.0, 5.0], [L + 1.5, L - 0.3, 0.2], [5.0, -9.0, 5.0], [4.9, 5.1, L + 2.0],
                    [0.1, 0.2, 0.3]])
    sig = np.array([0.8, 0.9, 0.7, 1.0, 0.6])
    got, ref = _project(grid, h, False, pos, sig, numax, cube, 16, "tf32", 605, storage)
    assert np.all(got[2] == 0.0)
    keep = [0, 1, 3, 4]
    assert_coeff_close(got[keep], ref[keep], TOL["tf32"])


@pytest.mark.parametrize("numax", list(range(8)))
def test_every_numax(numax):
    require_gpu()
    rng = np.random.default_rng(606 + numax)
    grid, h, cube = (40, 36, 32), 0.2, 16
    pos, sig = workloads.random_atoms(rng, 6, tuple(n * h for n in grid), True, min_sep=1.0)
    for prec in ("fp32", "tf32"):
        got, ref = _project(grid, h, True, pos, sig, numax, cube, 12, prec, 620 + numax)
        assert_coeff_close(got, ref, _tol(prec))
    for prec in ("fp32", "split_fp16"):
        got, ref = _project(grid, h, True, pos, sig, numax, cube, 24, prec, 640 + numax, "bf16")
        assert_coeff_close(got, ref, _tol(prec))


def test_plane_path_selection():
    """Eligible calls take the plane sweep (FP32 or BF16 rows of whole 16-byte units); a row longer than
    one TMA box (Nx > 256), unaligned band counts and numax 8 take the per-atom kernels; all give the
    oracle's result."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(630)
    h, numax, cube = 0.2, 3, 16
    psi = torch.zeros((40, 40, 40, 8), dtype=torch.float32, device="cuda")
    assert api.project_path(psi, numax, cube, h, True, "tf32") == "plane"
    assert api.project_path(psi, numax, cube, h, True, "fp32") == "plane"
    assert api.project_path(psi, 8, cube, h, True, "fp32") == "atom"
    assert api.project_path(psi.to(torch.bfloat16), numax, cube, h, True, "tf32") == "plane"
    assert api.project_path(psi[..., :4].contiguous().to(torch.bfloat16), numax, cube, h, True, "tf32") == "atom"
    assert api.project_path(torch.zeros((40, 40, 40, 6), device="cuda"), numax, cube, h, True, "tf32") == "atom"
    assert api.project_path(psi.double(), numax, cube, h, True, "ff64") == "atom"
    wide = (264, 16, 16)
    psi2 = rng.standard_normal((16, 16, 264, 4)).astype(np.float32)
    psi2_d = torch.from_numpy(psi2).cuda()
    assert api.project_path(psi2_d, numax, cube, h, True, "fp32") == "atom"
    pos2, sig2 = workloads.random_atoms(rng, 3, tuple(n * h for n in wide), True, min_sep=1.0)
    got = api.project(psi2_d, pos2, sig2, numax, cube, h, True, prec="fp32").double().cpu().numpy()
    ref = oracle.project(wide, h, True, psi2.astype(np.float64), pos2, sig2, numax, cube)
    assert_coeff_close(got, ref, TOL_FP32)


def test_plane_sweep_repeatable_and_status_clear():
    """Two calls give bit-identical coefficients (fixed plan, no atomics) and no bounded wait expired."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(640)
    grid, h, numax, cube = (64, 64, 64), 0.2, 7, 32
    pos, sig = workloads.random_atoms(rng, 40, tuple(n * h for n in grid), True, min_sep=1.5)
    psi = torch.from_numpy(rng.standard_normal((64, 64, 64, 64)).astype(np.float32)).cuda()
    hd = api.Handle(0)
    c1 = api.project(psi, pos, sig, numax, cube, h, True, prec="tf32", handle=hd)
    c2 = api.project(psi, pos, sig, numax, cube, h, True, prec="tf32", handle=hd)
    hd.sync()
    assert torch.equal(c1, c2)
    ref = oracle.project(grid, h, True, psi.double().cpu().numpy(), pos[:3], sig[:3], numax, cube)
    assert rel_norm(c1[:3].double().cpu().numpy(), ref) <= TOL["tf32"]


def _expand(grid, h, periodic, pos, sig, numax, cube, nbands, prec, seed):
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(seed)
    psi = rng.standard_normal((grid[2], grid[1], grid[0], nbands)).astype(np.float32)
    c = rng.standard_normal((len(pos), oracle.nstates(numax), nbands)).astype(np.float32)
    out = torch.from_numpy(psi).cuda()
    api.add(out, torch.from_numpy(c).cuda(), pos, sig, numax, cube, h, periodic, prec=prec)
    ref = oracle.add(grid, h, periodic, psi.astype(np.float64), pos, sig, numax, cube, c.astype(np.float64))
    return out.double().cpu().numpy() - psi, ref - psi


@pytest.mark.parametrize("prec", ["fp32", "tf32", "3xtf32", "bf16", "split_fp16"])
def test_expand_dense_atoms(prec):
    """Dense overlap: about 53 cubes meet each grid row."""
    require_gpu()
    rng = np.random.default_rng(611)
    grid, h, numax, cube = (48, 48, 48), 0.2, 3, 32
    pos, sig = workloads.random_atoms(rng, 120, tuple(n * h for n in grid), True, min_sep=0.6)
    got, ref = _expand(grid, h, True, pos, sig, numax, cube, 8, prec, 612)
    assert rel_norm(got, ref) <= _tol(prec)


@pytest.mark.parametrize("prec", ["fp32", "tf32", "split_fp16"])
def test_expand_wrapped_and_open(prec):
    require_gpu()
    rng = np.random.default_rng(613)
    grid, h, numax, cube = (36, 34, 40), 0.2, 5, 32
    pos, sig = workloads.random_atoms(rng, 7, tuple(n * h for n in grid), True, min_sep=1.0)
    got, ref = _expand(grid, h, True, pos, sig, numax, cube, 36, prec, 614)
    assert rel_norm(got, ref) <= _tol(prec)
    grid, h, numax = (40, 40, 40), 0.25, 4
    L = 40 * h
    pos = np.array([[-2.0, 3.0, 5.0], [L + 1.5, L - 0.3, 0.2], [5.0, -9.0, 5.0], [4.9, 5.1, L + 2.0], [0.1, 0.2, 0.3]])
    sig = np.array([0.8, 0.9, 0.7, 1.0, 0.6])
    got, ref = _expand(grid, h, False, pos, sig, numax, cube, 16, prec, 615)
    assert rel_norm(got, ref) <= _tol(prec)


@pytest.mark.parametrize("numax", list(range(8)))
def test_expand_every_numax(numax):
    require_gpu()
    rng = np.random.default_rng(616 + numax)
    grid, h, cube = (40, 36, 32), 0.2, 16
    pos, sig = workloads.random_atoms(rng, 6, tuple(n * h for n in grid), True, min_sep=1.0)
    for prec in ("fp32", "tf32", "bf16"):
        got, ref = _expand(grid, h, True, pos, sig, numax, cube, 12, prec, 640 + numax)
        assert rel_norm(got, ref) <= _tol(prec)


def test_expand_bitwise_repeatable():
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(650)
    grid, h, numax, cube = (64, 64, 64), 0.2, 7, 32
    pos, sig = workloads.random_atoms(rng, 40, tuple(n * h for n in grid), True, min_sep=1.5)
    c = torch.from_numpy(rng.standard_normal((40, oracle.nstates(numax), 64)).astype(np.float32)).cuda()
    outs = []
    for _ in range(2):
        out = torch.zeros((64, 64, 64, 64), dtype=torch.float32, device="cuda")
        api.add(out, c, pos, sig, numax, cube, h, True, prec="tf32")
        outs.append(out)
    assert torch.equal(outs[0], outs[1])


def test_plan_cache_follows_the_geometry():
    """The handle keeps the plan of the last geometry: alternating atom sets on one handle must each get
    their own plan (results equal to fresh-handle results, bit for bit)."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(660)
    grid, h, numax, cube = (48, 48, 48), 0.2, 5, 32
    box = tuple(n * h for n in grid)
    pa, sa = workloads.random_atoms(rng, 12, box, True, min_sep=1.0)
    pb, sb = workloads.random_atoms(rng, 9, box, True, min_sep=1.0)
    psi = torch.from_numpy(rng.standard_normal((48, 48, 48, 32)).astype(np.float32)).cuda()
    ref_a = api.project(psi, pa, sa, numax, cube, h, True, prec="tf32", handle=api.Handle(0))
    ref_b = api.project(psi, pb, sb, numax, cube, h, True, prec="tf32", handle=api.Handle(0))
    hd = api.Handle(0)
    for pos, sig, ref in ((pa, sa, ref_a), (pb, sb, ref_b), (pa, sa, ref_a), (pa, sa, ref_a)):
        got = api.project(psi, pos, sig, numax, cube, h, True, prec="tf32", handle=hd)
        assert torch.equal(got, ref)
    moved = pa.copy()
    moved[3, 1] += 0.37
    got = api.project(psi, moved, sa, numax, cube, h, True, prec="tf32", handle=hd).double().cpu().numpy()
    exp = oracle.project(grid, h, True, psi.double().cpu().numpy(), moved, sa, numax, cube)
    assert_coeff_close(got, exp, TOL["tf32"])


def test_plan_caches_survive_each_other():
    """One handle alternating FP32-class projections whose plane plan grows and expansions / generic
    projections whose geometry plans are cached: each cache keeps its own buffers (regression test)."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(670)
    grid, h, numax, cube = (48, 48, 48), 0.2, 3, 32
    box = tuple(n * h for n in grid)
    hd = api.Handle(0)
    psi32 = torch.from_numpy(rng.standard_normal((48, 48, 48, 8)).astype(np.float32)).cuda()
    psi64 = psi32.double()
    small, ssig = workloads.random_atoms(rng, 4, box, True, min_sep=1.0)
    big, bsig = workloads.random_atoms(rng, 60, box, True, min_sep=0.8)
    c_small = torch.from_numpy(rng.standard_normal((4, 20, 8)).astype(np.float32)).cuda()
    ref = oracle.add(grid, h, True, np.zeros((48, 48, 48, 8)), small, ssig, numax, cube, c_small.double().cpu().numpy())
    for _ in range(2):
        out = torch.zeros_like(psi32)
        api.add(out, c_small, small, ssig, numax, cube, h, True, prec="fp32", handle=hd)  # geometry cache
        api.project(psi64, small, ssig, numax, cube, h, True, prec="fp64", handle=hd)     # geometry cache
        api.project(psi32, big, bsig, numax, cube, h, True, prec="tf32", handle=hd)       # plane plan grows
        out2 = torch.zeros_like(psi32)
        api.add(out2, c_small, small, ssig, numax, cube, h, True, prec="fp32", handle=hd)  # cached geometry
        assert rel_norm(out2.double().cpu().numpy(), ref) <= TOL_FP32
        assert torch.equal(out, out2)
