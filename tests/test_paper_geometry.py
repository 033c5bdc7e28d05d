"""The paper's benchmark geometry (Sec. 6) is reproduced by the workload generator (CPU)."""
import os

import numpy as np

import workloads

GOLDEN = os.path.join(os.path.dirname(__file__), "golden", "fcc_geometry.txt")


def _golden():
    vals = {}
    with open(GOLDEN) as fh:
        for line in fh:
            if line.strip() and not line.startswith("#"):
                k, v = line.split()
                vals[k] = int(v)
    return vals


def test_fcc_geometry_matches_printed_counts():
    g = _golden()
    grid, h, pos, sig = workloads.fcc_paper_geometry()
    assert grid == (g["grid_points_per_axis"],) * 3
    assert len(pos) == g["atoms_touching"]
    assert abs(h - 0.25 * workloads.ANGSTROM) < 1e-12
    # nearest-neighbour distance a / sqrt(2) = 2.885 A (the paper quotes 2.9 A)
    d = np.linalg.norm(pos[:, None, :] - pos[None, :, :], axis=-1)
    d[np.diag_indices_from(d)] = np.inf
    assert abs(d.min() / workloads.ANGSTROM - 4.08 / np.sqrt(2)) < 1e-9
    # the cube of edge 32 points (15.1 Bohr) holds each 3.55 A projection sphere
    assert 32 * h / 2 > 3.55 * workloads.ANGSTROM
