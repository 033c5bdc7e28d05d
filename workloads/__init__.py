"""Seeded synthetic inputs shared by the tests, the smoke check and the benchmark.

This module draws random numbers and shapes only: it holds none of the projection arithmetic, so the
oracle and the CUDA path can both consume its arrays without sharing code.  Basis sizes are passed in
by the caller.

Workload shapes follow the paper's setting (real-space grid wave functions, bands innermost, atoms
with a width sigma each; Sec. 3.2 and Sec. 6) at the sizes of the five named configurations:

  tiny    16^3 grid (= the cube), h = 0.25, 1 atom at (7.37, 7.52, 7.18) h, sigma 1.0, numax 3,
          cube 16, 4 bands N(0,1), FP64, not periodic
  c96     periodic 96^3, h = 0.2, 64 atoms uniform (min image separation 2.0), sigma U[0.5, 1.0],
          numax 5, cube 32, 128 bands N(0,1) FP64; expansion coefficients N(0,1) FP64
  c160    periodic 160^3, h = 0.2, 512 atoms (min separation 2.0), sigma U[0.5, 1.0], numax 7, cube 32,
          256 bands N(0,1) stored FP32 / BF16
  c128    periodic 128^3, h = 0.2, 128 atoms (min separation 2.0), sigma U[0.5, 1.0], numax 5, cube 32,
          64 bands N(0,1) FP32; D ~ U[-1, 1] per (atom, state)
  serve   systems with grid 48^3..192^3 (step 16), h = 0.2, cube 32, atoms log-uniform in
          [8, min(1024, 0.05 L^3)], bands log-uniform in [16, 512] (multiple of 16), numax in {3,5,7,9}
"""
from __future__ import annotations

import dataclasses
import math

import numpy as np

SEED_BASE = 1000


@dataclasses.dataclass(frozen=True)
class Workload:
    name: str
    grid: tuple          # (Nx, Ny, Nz)
    h: float
    periodic: bool
    natoms: int
    numax: int
    cube: int
    nbands: int
    dtype: str           # storage type of psi: "f64" | "f32" | "bf16"
    seed: int
    min_sep: float = 2.0
    sigma_range: tuple = (0.5, 1.0)
    fixed_pos: tuple = None     # explicit atom positions (Bohr) for the tiny case
    fixed_sigma: tuple = None

    @property
    def box(self):
        return tuple(n * self.h for n in self.grid)


WORKLOADS = {
    "tiny": Workload("tiny", (16, 16, 16), 0.25, False, 1, 3, 16, 4, "f64", SEED_BASE + 1,
                     fixed_pos=((7.37 * 0.25, 7.52 * 0.25, 7.18 * 0.25),), fixed_sigma=(1.0,)),
    "c96": Workload("c96", (96, 96, 96), 0.2, True, 64, 5, 32, 128, "f64", SEED_BASE + 2),
    "c160": Workload("c160", (160, 160, 160), 0.2, True, 512, 7, 32, 256, "f32", SEED_BASE + 3),
    "c128": Workload("c128", (128, 128, 128), 0.2, True, 128, 5, 32, 64, "f32", SEED_BASE + 4),
}


def rng_for(w: Workload, stream: int = 0) -> np.random.Generator:
    return np.random.default_rng([w.seed, stream])


def atoms(w: Workload, rng: np.random.Generator = None):
    """Atom positions [A][3] (Bohr, inside the box) and widths sigma [A], both float64.

    Positions are uniform in the box, rejection-sampled so that every pair is at least ``min_sep``
    apart (minimum-image distance when periodic)."""
    if w.fixed_pos is not None:
        return (np.array(w.fixed_pos, dtype=np.float64).reshape(-1, 3),
                np.array(w.fixed_sigma, dtype=np.float64).reshape(-1))
    rng = rng if rng is not None else rng_for(w, 0)
    return random_atoms(rng, w.natoms, w.box, w.periodic, w.min_sep, w.sigma_range)


def random_atoms(rng, natoms, box, periodic, min_sep=2.0, sigma_range=(0.5, 1.0), max_tries=200000):
    box = np.asarray(box, dtype=np.float64)
    pos = np.zeros((natoms, 3), dtype=np.float64)
    count, tries = 0, 0
    while count < natoms:
        tries += 1
        if tries > max_tries:
            raise RuntimeError(f"could not place {natoms} atoms with separation {min_sep} in box {box}")
        cand = rng.uniform(0.0, 1.0, size=3) * box
        if count:
            d = pos[:count] - cand
            if periodic:
                d -= box * np.round(d / box)
            if np.min(np.einsum("ij,ij->i", d, d)) < min_sep * min_sep:
                continue
        pos[count] = cand
        count += 1
    sigma = rng.uniform(sigma_range[0], sigma_range[1], size=natoms).astype(np.float64)
    return pos, sigma


def psi_host(w: Workload, rng: np.random.Generator = None, nbands: int = None) -> np.ndarray:
    """Wave functions psi[Nz][Ny][Nx][B] ~ N(0,1), float64, drawn on the host."""
    rng = rng if rng is not None else rng_for(w, 1)
    nb = w.nbands if nbands is None else nbands
    nx, ny, nz = w.grid
    return rng.standard_normal((nz, ny, nx, nb))


def coeff_host(w: Workload, nstates: int, rng: np.random.Generator = None, nbands: int = None) -> np.ndarray:
    """Expansion coefficients c[A][N][B] ~ N(0,1), float64 (N given by the caller)."""
    rng = rng if rng is not None else rng_for(w, 2)
    nb = w.nbands if nbands is None else nbands
    return rng.standard_normal((w.natoms, nstates, nb))


def dmatrix_host(w: Workload, nstates: int, rng: np.random.Generator = None) -> np.ndarray:
    """Per-(atom, state) weights D ~ U[-1, 1] for the energy E = sum D c^2."""
    rng = rng if rng is not None else rng_for(w, 3)
    return rng.uniform(-1.0, 1.0, size=(w.natoms, nstates))


def psi_device(w: Workload, torch_dtype=None, device="cuda", nbands: int = None):
    """psi[Nz][Ny][Nx][B] ~ N(0,1) drawn on the device with torch's seeded Philox generator (for sizes
    too large to draw on the host quickly).  Returned in the workload's storage dtype."""
    import torch
    g = torch.Generator(device=device)
    g.manual_seed(w.seed)
    nx, ny, nz = w.grid
    nb = w.nbands if nbands is None else nbands
    dt = torch_dtype or {"f64": torch.float64, "f32": torch.float32, "bf16": torch.bfloat16}[w.dtype]
    gen_dt = torch.float64 if dt == torch.float64 else torch.float32
    x = torch.randn((nz, ny, nx, nb), generator=g, device=device, dtype=gen_dt)
    return x.to(dt)


# ---------------------------------------------------------------------------------------------------
# the paper's benchmark geometry (Sec. 6)

ANGSTROM = 1.0 / 0.52917721092   # Bohr per Angstrom


def fcc_paper_geometry(lattice_A=4.08, box_A=16.0, h_A=0.25, rprj_A=3.55, sigma_bohr=0.59):
    """The benchmark system of Sec. 6: a cubic domain of 16 A edge sampled at 0.25 A (64^3 points),
    fcc lattice with a = 4.08 A anchored at the domain corner, and every atom whose projection sphere
    (3.55 A) overlaps the domain.  Returns (grid, h, positions [A][3], sigma [A]) in Bohr; sigma is the
    0.59 Bohr the paper selects for Pt (Sec. 4).  Not periodic."""
    n = int(round(box_A / h_A))
    a = lattice_A
    basis = np.array([[0, 0, 0], [0.5, 0.5, 0], [0.5, 0, 0.5], [0, 0.5, 0.5]])
    lo, hi = int(np.floor(-rprj_A / a)) - 1, int(np.ceil((box_A + rprj_A) / a)) + 1
    pts = []
    for i in range(lo, hi + 1):
        for j in range(lo, hi + 1):
            for k in range(lo, hi + 1):
                for b in basis:
                    p = (np.array([i, j, k]) + b) * a
                    d = np.maximum(0.0, np.maximum(-p, p - box_A))
                    if np.sqrt(np.dot(d, d)) < rprj_A:
                        pts.append(p)
    pos = np.array(pts, dtype=np.float64) * ANGSTROM
    return (n, n, n), h_A * ANGSTROM, pos, np.full(len(pos), sigma_bohr)


# ---------------------------------------------------------------------------------------------------
# serving stream


@dataclasses.dataclass(frozen=True)
class SystemSpec:
    grid: int          # cubic grid edge (points)
    natoms: int
    nbands: int
    numax: int
    seed: int
    h: float = 0.2
    cube: int = 32
    periodic: bool = True


def serving_systems(count: int, seed: int = SEED_BASE + 5, max_grid: int = 192, max_bands: int = 512,
                    max_atoms: int = 1024, numaxes=(3, 5, 7, 9)):
    """Draw ``count`` heterogeneous systems for the serving stream (sizes as in the module docstring;
    atoms are capped at 0.05 L^3 so the separation constraint can be met)."""
    rng = np.random.default_rng(seed)
    grids = list(range(48, max_grid + 1, 16))
    out = []
    for i in range(count):
        g = int(rng.choice(grids))
        L = g * 0.2
        amax = max(8, min(max_atoms, int(0.05 * L ** 3)))
        na = int(round(math.exp(rng.uniform(math.log(8), math.log(amax)))))
        nb = int(round(math.exp(rng.uniform(math.log(16), math.log(max_bands))) / 16.0)) * 16
        nb = max(16, min(max_bands, nb))
        nu = int(rng.choice(numaxes))
        out.append(SystemSpec(grid=g, natoms=na, nbands=nb, numax=nu, seed=seed * 1000 + i))
    return out


def poisson_arrivals(rng: np.random.Generator, count: int, rate_per_s: float) -> np.ndarray:
    """Arrival times (s) of a Poisson stream."""
    return np.cumsum(rng.exponential(1.0 / rate_per_s, size=count))
