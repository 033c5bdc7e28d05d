"""The seeded synthetic inputs follow their stated recipe (CPU): sizes of the named workloads, atoms
inside the box at a minimum (minimum-image) separation of 2.0, sigma in [0.5, 1.0], reproducibility from
the seed, the serving systems' ranges, and the paper's fcc benchmark geometry."""
import numpy as np
import pytest

import workloads


def _min_image_distance(pos, box, periodic):
    d = pos[:, None, :] - pos[None, :, :]
    if periodic:
        d -= box * np.round(d / box)
    r = np.sqrt(np.einsum("ijk,ijk->ij", d, d))
    r[np.diag_indices(len(pos))] = np.inf
    return r.min()


@pytest.mark.parametrize("name,grid,natoms,numax,bands", [("c96", 96, 64, 5, 128), ("c160", 160, 512, 7, 256),
                                                        ("c128", 128, 128, 5, 64)])
def test_named_workloads(name, grid, natoms, numax, bands):
    w = workloads.WORKLOADS[name]
    assert w.grid == (grid,) * 3 and w.h == 0.2 and w.periodic and w.cube == 32
    assert (w.natoms, w.numax, w.nbands) == (natoms, numax, bands)
    pos, sig = workloads.atoms(w)
    box = np.array(w.box)
    assert pos.shape == (natoms, 3) and np.all(pos >= 0) and np.all(pos < box)
    assert _min_image_distance(pos, box, True) >= 2.0
    assert np.all((sig >= 0.5) & (sig <= 1.0))
    pos2, sig2 = workloads.atoms(w)
    assert np.array_equal(pos, pos2) and np.array_equal(sig, sig2)   # seeded


def test_tiny_case_is_the_stated_single_atom():
    w = workloads.WORKLOADS["tiny"]
    pos, sig = workloads.atoms(w)
    assert np.allclose(pos[0] / w.h, [7.37, 7.52, 7.18]) and sig[0] == 1.0
    o = np.floor(pos[0] / w.h).astype(int) - w.cube // 2 + 1
    assert np.array_equal(o, [0, 0, 0])   # the cube is the grid


def test_serving_systems_ranges():
    systems = workloads.serving_systems(40)
    for s in systems:
        assert 48 <= s.grid <= 192 and s.grid % 16 == 0
        assert 8 <= s.natoms <= min(1024, max(8, int(0.05 * (s.grid * 0.2) ** 3)))
        assert 16 <= s.nbands <= 512 and s.nbands % 16 == 0
        assert s.numax in (3, 5, 7, 9)
    assert len({s.numax for s in systems}) > 1 and len({s.grid for s in systems}) > 1


def test_paper_fcc_geometry_shape():
    grid, h, pos, sig = workloads.fcc_paper_geometry()
    assert grid == (64, 64, 64) and abs(h - 0.25 * workloads.ANGSTROM) < 1e-12
    assert pos.shape == (665, 3) and np.all(sig == 0.59)
