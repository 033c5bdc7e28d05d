"""Library Cartesian <-> radial transform (eq. SHO-transform-Cartesian-to-radial, Sec. 2.4) against the
oracle: the host-built U (exact polynomial algebra) against the oracle's quadrature U on the CPU, and the
device transform against the oracle's matrix product on the GPU."""
import numpy as np
import pytest

import oracle
import workloads
from helpers import TOL_FP64, rel_norm, require_gpu
from oracle import radial


@pytest.mark.parametrize("numax", list(range(10)))
def test_library_matrix_matches_oracle(numax):
    from paper_1905_00480_gb300 import api
    assert api.radial_labels(numax) == radial.radial_labels(numax)
    U = api.radial_matrix(numax)
    ref = radial.radial_matrix(numax)
    assert np.max(np.abs(U - ref)) < 1e-12


def test_library_rejects_bad_numax():
    from paper_1905_00480_gb300 import api, ShoError
    with pytest.raises(ShoError):
        api.radial_matrix(10)


@pytest.mark.gpu
@pytest.mark.parametrize("numax", [0, 3, 5, 7, 9])
def test_device_transform(numax):
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    rng = np.random.default_rng(700 + numax)
    A, B = 5, 45
    c = rng.standard_normal((A, oracle.nstates(numax), B))
    cd = torch.from_numpy(c).cuda()
    got = api.to_radial(cd, numax).cpu().numpy()
    ref = radial.to_radial(c, numax)
    assert rel_norm(got, ref) <= TOL_FP64
    back = api.to_radial(torch.from_numpy(got).cuda(), numax, inverse=True).cpu().numpy()
    assert rel_norm(back, c) <= TOL_FP64
    got32 = api.to_radial(cd.float(), numax).double().cpu().numpy()
    assert rel_norm(got32, radial.to_radial(cd.float().double().cpu().numpy(), numax)) <= 2e-6


@pytest.mark.gpu
def test_projected_radial_state_is_a_unit_vector():
    """A radial state sampled on a fine grid, projected by the GPU (FP64) and transformed on the GPU, is
    the unit vector of that state (the oracle-side version of this check is a CPU pin)."""
    require_gpu()
    import torch
    from paper_1905_00480_gb300 import api
    numax, sigma, h, C = 4, 0.42, 0.1, 64
    X = np.array([[C * h / 2 + 0.013, C * h / 2 - 0.021, C * h / 2 + 0.007]])
    j = np.arange(C) * h
    xx, yy, zz = np.meshgrid(j - X[0, 0], j - X[0, 1], j - X[0, 2], indexing="ij")
    labels = radial.radial_labels(numax)
    states = [0, 5, 14, 20, 34]
    psi = np.stack([np.transpose(radial.radial_value(*labels[s], xx, yy, zz, sigma), (2, 1, 0)) for s in states],
                   axis=-1)
    c = api.project(torch.from_numpy(np.ascontiguousarray(psi)).cuda(), X, [sigma], numax, C, h, False, prec="fp64")
    crad = api.to_radial(c, numax).cpu().numpy()[0]
    for i, s in enumerate(states):
        e = np.zeros(len(labels))
        e[s] = 1.0
        assert np.max(np.abs(crad[:, i] - e)) < 1e-9, labels[s]
