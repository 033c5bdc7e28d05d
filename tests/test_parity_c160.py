"""The precision workload at full size (GPU): 160^3 periodic grid, h = 0.2, 512 atoms, numax 7 (120
states), cube 32, 256 bands, psi stored FP32 and BF16, every FP32-class form, in the launch configuration
the benchmark times.

The oracle cannot run the whole workload in seconds, so it checks samples: the projection of 6 seeded
atoms (norm-wise per atom and max-wise) and the expansion at 400 seeded grid points, both against the
FP64 oracle run on the storage-rounded inputs the kernels see.  Bars, per form, from the operand rounding
of its x-pass (u = unit roundoff of the operand type; see tests/test_parity_tc.py):
  FP32 (CUDA cores)      TOL_FP32 = 2e-6
  TF32                   2e-3    (u = 2^-11)
  3XTF32, SPLIT_FP16     1e-5    (22 operand bits)
  BF16                   1.5e-2  (u = 2^-8)
BF16-stored expansion results are rounded once to BF16 on store: 2^-8 is added to the bar there.
"""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP32, rel_max, rel_norm, require_gpu

pytestmark = pytest.mark.gpu

TOL = {"fp32": TOL_FP32, "tf32": 2e-3, "3xtf32": 1e-5, "bf16": 1.5e-2, "split_fp16": 1e-5}
STORE_ROUND = {"f32": 0.0, "bf16": 2.0 ** -8}
FORMS = ["fp32", "tf32", "3xtf32", "bf16", "split_fp16"]


@pytest.fixture(scope="module")
def c160():
    """Atoms, sampled atoms / points and the expansion coefficients (FP32) of the 160^3 workload."""
    require_gpu()
    import torch
    w = workloads.WORKLOADS["c160"]
    pos, sig = workloads.atoms(w)
    N = oracle.nstates(w.numax)
    rng = np.random.default_rng(1603)
    sel = np.sort(rng.choice(w.natoms, size=6, replace=False))
    pts = np.sort(rng.choice(w.grid[0] * w.grid[1] * w.grid[2], size=400, replace=False))
    c_d = torch.from_numpy(workloads.coeff_host(w, N)).to("cuda", torch.float32)
    c_r = c_d.double().cpu().numpy()
    ref_add = oracle.expand_points(w.grid, w.h, w.periodic, pos, sig, w.numax, w.cube, c_r, pts)
    return dict(w=w, pos=pos, sig=sig, sel=sel, pts=pts, c_d=c_d, ref_add=ref_add)


@pytest.fixture(scope="module", params=["f32", "bf16"])
def stored(request, c160):
    """psi in one storage type on the device, and the oracle's projection of the sampled atoms on the
    storage-rounded values."""
    import torch
    w = c160["w"]
    tdt = {"f32": torch.float32, "bf16": torch.bfloat16}[request.param]
    psi_d = workloads.psi_device(w, torch_dtype=tdt)
    psi_r = psi_d.double().cpu().numpy()
    sel = c160["sel"]
    ref = oracle.project(w.grid, w.h, w.periodic, psi_r, c160["pos"][sel], c160["sig"][sel], w.numax, w.cube)
    del psi_r
    yield request.param, psi_d, ref
    del psi_d
    torch.cuda.empty_cache()


@pytest.mark.parametrize("form", FORMS)
def test_c160_projection_sampled_atoms(c160, stored, form):
    from paper_1905_00480_gb300 import api
    w = c160["w"]
    storage, psi_d, ref = stored
    got = api.project(psi_d, c160["pos"], c160["sig"], w.numax, w.cube, w.h, w.periodic, prec=form)
    got = got[c160["sel"]].double().cpu().numpy()
    for i in range(len(c160["sel"])):
        e = rel_norm(got[i], ref[i])
        assert e <= TOL[form], f"{storage}/{form} atom {c160['sel'][i]}: norm-wise {e:.3e} > {TOL[form]:.1e}"
    assert rel_max(got, ref) <= TOL[form]


@pytest.mark.parametrize("form", FORMS)
def test_c160_expansion_sampled_points(c160, stored, form):
    import torch
    from paper_1905_00480_gb300 import api
    w = c160["w"]
    storage, psi_d, _ = stored
    out = torch.zeros_like(psi_d)
    api.add(out, c160["c_d"], c160["pos"], c160["sig"], w.numax, w.cube, w.h, w.periodic, prec=form)
    idx = torch.from_numpy(c160["pts"]).cuda()
    got = out.reshape(-1, w.nbands).index_select(0, idx).double().cpu().numpy()
    del out
    tol = TOL[form] + STORE_ROUND[storage]
    e = rel_norm(got, c160["ref_add"])
    assert e <= tol, f"{storage}/{form}: norm-wise {e:.3e} > {tol:.1e}"
    assert rel_max(got, c160["ref_add"]) <= 2 * tol
