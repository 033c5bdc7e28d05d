"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics (CPU only).

Each test checks the oracle against something other than itself: values printed in the paper
(tests/golden/), textbook closed forms, the paper's own Hermite recursion evaluated in exact rational
arithmetic, independent library evaluations (scipy), integrals with closed forms, exact symmetries and
finite differences.  A dropped term, a wrong sign, a swapped index or a transposed operand in the oracle
fails at least one of them.
"""
import math
import os
from fractions import Fraction

import numpy as np
import pytest
from scipy import special

import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


# --------------------------------------------------------------------------- independent helpers
def _phi_scipy(n, u, sigma):
    """Normalised 1D oscillator function built from scipy's Hermite polynomial (independent of the
    oracle's power sum)."""
    xi = np.asarray(u, dtype=np.float64) / sigma
    norm = 1.0 / math.sqrt(sigma * math.sqrt(math.pi) * 2.0 ** n * math.factorial(n))
    return norm * special.eval_hermite(n, xi) * np.exp(-0.5 * xi * xi)


def _enumerate(numax):
    """(nx, ny, nz) list in the library's documented order: nz outer, ny middle, nx inner."""
    return [(nx, ny, nz) for nz in range(numax + 1) for ny in range(numax + 1 - nz)
            for nx in range(numax + 1 - nz - ny)]


def _brute_project(grid, h, periodic, psi, pos, sigma, numax, cube, rprj=0.0):
    """Direct definition with scipy functions and explicit loops (tiny inputs only); rprj > 0 keeps only
    the cube points inside the atom's sphere."""
    nx_, ny_, nz_ = grid
    states = _enumerate(numax)
    B = psi.shape[-1]
    out = np.zeros((len(pos), len(states), B))
    for a, (X, s) in enumerate(zip(pos, sigma)):
        o = [math.floor(X[d] / h) - cube // 2 + 1 for d in range(3)]
        for iz in range(cube):
            for iy in range(cube):
                for ix in range(cube):
                    j = [o[0] + ix, o[1] + iy, o[2] + iz]
                    if periodic:
                        j = [j[0] % nx_, j[1] % ny_, j[2] % nz_]
                    elif not (0 <= j[0] < nx_ and 0 <= j[1] < ny_ and 0 <= j[2] < nz_):
                        continue
                    u = [(o[0] + ix) * h - X[0], (o[1] + iy) * h - X[1], (o[2] + iz) * h - X[2]]
                    if rprj > 0 and not (u[0] * u[0] + u[1] * u[1]) + u[2] * u[2] <= rprj * rprj:
                        continue
                    for k, (mx, my, mz) in enumerate(states):
                        w = _phi_scipy(mx, u[0], s) * _phi_scipy(my, u[1], s) * _phi_scipy(mz, u[2], s)
                        out[a, k] += h ** 3 * w * psi[j[2], j[1], j[0]]
    return out


def _sample_state(grid, h, X, sigma, m):
    """psi = Psi_m sampled on the whole (non-periodic) grid, [Nz][Ny][Nx][1]."""
    nx_, ny_, nz_ = grid
    fx = _phi_scipy(m[0], np.arange(nx_) * h - X[0], sigma)
    fy = _phi_scipy(m[1], np.arange(ny_) * h - X[1], sigma)
    fz = _phi_scipy(m[2], np.arange(nz_) * h - X[2], sigma)
    return np.einsum("z,y,x->zyx", fz, fy, fx)[..., None]


# --------------------------------------------------------------------------- 1. basis size
def test_state_count_matches_paper_table():
    with open(os.path.join(GOLDEN, "state_counts.txt")) as fh:
        rows = [l.split() for l in fh if l.strip() and l[0] != "#"]
    assert rows, "golden file empty"
    for nu, count in rows:
        assert oracle.nstates(int(nu)) == int(count)
        assert len(oracle.basis(int(nu))) == int(count)


def test_basis_enumeration_order_and_completeness():
    for nu in range(0, 11):
        b = oracle.basis(nu)
        assert [tuple(r) for r in b] == _enumerate(nu)
        assert len({tuple(r) for r in b}) == len(b)
        assert (b.sum(axis=1) <= nu).all()


# --------------------------------------------------------------------------- 2. Hermite polynomials
TEXTBOOK_H = {  # physicists' Hermite polynomials, textbook closed forms
    0: lambda x: 1.0,
    1: lambda x: 2 * x,
    2: lambda x: 4 * x ** 2 - 2,
    3: lambda x: 8 * x ** 3 - 12 * x,
    4: lambda x: 16 * x ** 4 - 48 * x ** 2 + 12,
    5: lambda x: 32 * x ** 5 - 160 * x ** 3 + 120 * x,
}


@pytest.mark.parametrize("n", sorted(TEXTBOOK_H))
def test_hermite_textbook_closed_forms(n):
    for x in (-2.3, -0.7, 0.0, 0.31, 1.0, 1.9, 3.7):
        ref = TEXTBOOK_H[n](x)
        assert abs(oracle.hermite(n, x) - ref) <= 1e-14 * max(1.0, abs(ref))


def test_hermite_matches_paper_monic_recursion_exactly():
    """Sec. 3.7: h_0 = 1, h_1 = x, h_{n+1} = x h_n - (n/2) h_{n-1} (monic), i.e. H_n = 2^n h_n.  The
    recursion is run here in exact rational arithmetic."""
    for x in (Fraction(-17, 7), Fraction(3, 10), Fraction(5, 2), Fraction(41, 8)):
        hm, h0 = Fraction(0), Fraction(1)
        for n in range(0, 13):
            exact = (2 ** n) * h0
            got = oracle.hermite(n, float(x))
            assert abs(got - float(exact)) <= 1e-13 * max(1.0, abs(float(exact))), (n, x)
            hm, h0 = h0, x * h0 - Fraction(n, 2) * hm


def test_monic_closed_forms_from_recursion():
    """h2 = x^2 - 1/2, h3 = x^3 - 3x/2, h4 = x^4 - 3x^2 + 3/4 (the recursion of Sec. 3.7 unrolled)."""
    for x in (-1.3, 0.4, 2.2):
        assert abs(oracle.hermite(2, x) / 4 - (x * x - 0.5)) < 1e-14
        assert abs(oracle.hermite(3, x) / 8 - (x ** 3 - 1.5 * x)) < 1e-13
        assert abs(oracle.hermite(4, x) / 16 - (x ** 4 - 3 * x * x + 0.75)) < 1e-13


def test_phi_matches_scipy_construction():
    for n in range(0, 12):
        for s in (0.5, 0.77, 1.0):
            for u in (-2.9, -0.33, 0.0, 0.6, 1.7, 3.1):
                ref = float(_phi_scipy(n, u, s))
                assert abs(oracle.phi(n, u, s) - ref) <= 1e-13 * max(1e-3, abs(ref))


# --------------------------------------------------------------------------- 3. 1D eigen-equation
@pytest.mark.parametrize("n", [0, 1, 2, 5, 9])
def test_phi_solves_oscillator_equation(n):
    """eq. 1HO_Hamiltonian: -phi'' + x^2 sigma^-4 phi = (2n+1) sigma^-2 phi (Sec. 2.2)."""
    s, d = 0.8, 1e-4
    for u in (-1.1, -0.4, 0.25, 0.9, 1.6):
        d2 = (oracle.dphi(n, u + d, s) - oracle.dphi(n, u - d, s)) / (2 * d)
        lhs = -d2 + u * u / s ** 4 * oracle.phi(n, u, s)
        rhs = (2 * n + 1) / s ** 2 * oracle.phi(n, u, s)
        scale = max(abs(rhs), (2 * n + 1) / s ** 2 * 1e-3)
        assert abs(lhs - rhs) <= 1e-6 * scale


def test_dphi_matches_finite_difference():
    s, d = 0.63, 1e-5
    for n in range(0, 10):
        for u in (-1.3, 0.0, 0.77, 2.0):
            fd = (oracle.phi(n, u + d, s) - oracle.phi(n, u - d, s)) / (2 * d)
            assert abs(oracle.dphi(n, u, s) - fd) <= 1e-8 * max(1.0, abs(fd))


def test_phi_orthonormal_1d_quadrature():
    from scipy import integrate
    s = 0.7
    for n in range(0, 8):
        for m in range(0, 8):
            val, _ = integrate.quad(lambda u: oracle.phi(n, u, s) * oracle.phi(m, u, s), -12 * s, 12 * s,
                                    limit=400, epsabs=1e-14)
            assert abs(val - (1.0 if n == m else 0.0)) < 1e-11


# --------------------------------------------------------------------------- 4. 3D projections
def test_eigenstate_projects_to_unit_vector():
    """A sampled SHO state projects to the unit vector of its index (Sec. 2.5 completeness / the
    truncated projector), with a wide cube and h <= h_max/2 (eq. max_grid_spacing)."""
    h, sigma, numax, cube = 0.2, 0.9, 4, 64
    grid = (64, 64, 64)
    X = np.array([[6.37, 6.52, 6.18]])
    hmax = math.pi * sigma / math.sqrt(2 * numax + 1)
    assert h <= hmax / 2
    states = _enumerate(numax)
    for m in [(0, 0, 0), (1, 0, 0), (0, 2, 1), (3, 0, 1), (1, 1, 2)]:
        psi = _sample_state(grid, h, X[0], sigma, m)
        c = oracle.project(grid, h, False, psi, X, [sigma], numax, cube)[0, :, 0]
        e = np.zeros(len(states))
        e[states.index(m)] = 1.0
        assert np.max(np.abs(c - e)) < 1e-12, (m, np.max(np.abs(c - e)))


def test_constant_psi_closed_form():
    """psi = 1: c_{nx ny nz} = prod_d integral(phi_{n_d}); odd n vanish, even n = 2m give
    sqrt(2 sigma) pi^(1/4) sqrt((2m)!)/(2^m m!) per axis (Gaussian integrals of Hermite functions)."""
    h, sigma, numax, cube = 0.2, 0.6, 5, 64
    grid = (64, 64, 64)
    X = np.array([[6.41, 6.29, 6.35]])
    psi = np.ones((64, 64, 64, 1))
    c = oracle.project(grid, h, False, psi, X, [sigma], numax, cube)[0, :, 0]

    def one_axis(n):
        if n % 2:
            return 0.0
        m = n // 2
        return math.sqrt(2 * sigma) * math.pi ** 0.25 * math.sqrt(math.factorial(2 * m)) / (2 ** m * math.factorial(m))

    ref = np.array([one_axis(a) * one_axis(b) * one_axis(cc) for a, b, cc in _enumerate(numax)])
    assert abs(ref[0] - (2 * sigma) ** 1.5 * math.pi ** 0.75) < 1e-14
    assert np.max(np.abs(c - ref)) < 1e-12


def test_plane_wave_fourier_eigenfunction():
    """Sec. 3.6: Hermite functions are eigenfunctions of the Fourier transform, so for psi = e^{i q.r}
    the coefficients are e^{i q.X} prod_d sqrt(2 pi) i^{n_d} phi_{n_d}^{(1/sigma)}(q_d)."""
    h, sigma, numax, cube = 0.2, 0.75, 4, 64
    grid = (64, 64, 64)
    X = np.array([6.33, 6.47, 6.21])
    q = np.array([1.3, -0.6, 2.1])
    zz, yy, xx = np.meshgrid(np.arange(64) * h, np.arange(64) * h, np.arange(64) * h, indexing="ij")
    phase = q[0] * xx + q[1] * yy + q[2] * zz
    psi = np.stack([np.cos(phase), np.sin(phase)], axis=-1)
    c = oracle.project(grid, h, False, psi, X[None], [sigma], numax, cube)[0]
    cz = c[:, 0] + 1j * c[:, 1]

    def ft(n, qd):  # integral phi_n(u) e^{i q u} du
        return math.sqrt(2 * math.pi) * (1j ** n) * _phi_scipy(n, qd, 1.0 / sigma)

    ref = np.array([np.exp(1j * q @ X) * ft(a, q[0]) * ft(b, q[1]) * ft(cc, q[2]) for a, b, cc in _enumerate(numax)])
    assert np.max(np.abs(cz - ref)) < 1e-11


def test_brute_force_tiny_periodic_and_clipped():
    rng = np.random.default_rng(7)
    grid = (6, 7, 5)
    psi = rng.standard_normal((5, 7, 6, 2))
    pos = np.array([[0.13, 1.01, 0.77], [1.27, 0.05, 0.44]])
    sig = np.array([0.6, 0.9])
    for periodic in (True, False):
        ref = _brute_project(grid, 0.25, periodic, psi, pos, sig, 2, 4)
        got = oracle.project(grid, 0.25, periodic, psi, pos, sig, 2, 4)
        assert np.max(np.abs(got - ref)) < 1e-13 * np.max(np.abs(ref))


def test_adjoint_identity():
    """<P psi, c> = h^3 <psi, E c>: expansion is the adjoint of projection in the h^3-weighted grid
    inner product (projection carries the quadrature weight, expansion does not)."""
    rng = np.random.default_rng(11)
    grid, h = (20, 18, 22), 0.21
    pos = np.array([[1.1, 2.3, 0.2], [3.9, 0.4, 4.4], [2.0, 2.0, 2.1]])
    sig = np.array([0.55, 0.8, 0.7])
    numax, cube, B = 3, 12, 3
    psi = rng.standard_normal((22, 18, 20, B))
    for periodic in (True, False):
        c = rng.standard_normal((3, oracle.nstates(numax), B))
        lhs = np.sum(oracle.project(grid, h, periodic, psi, pos, sig, numax, cube) * c)
        Ec = oracle.add(grid, h, periodic, np.zeros_like(psi), pos, sig, numax, cube, c)
        rhs = h ** 3 * np.sum(psi * Ec)
        assert abs(lhs - rhs) < 1e-13 * (abs(lhs) + 1.0)


def test_expand_points_matches_add():
    rng = np.random.default_rng(3)
    grid, h = (16, 14, 18), 0.2
    pos = np.array([[0.3, 2.0, 1.1], [2.7, 0.1, 3.3]])
    sig = np.array([0.6, 0.95])
    numax, cube, B = 4, 10, 2
    c = rng.standard_normal((2, oracle.nstates(numax), B))
    full = oracle.add(grid, h, True, np.zeros((18, 14, 16, B)), pos, sig, numax, cube, c).reshape(-1, B)
    pts = rng.choice(full.shape[0], size=50, replace=False)
    got = oracle.expand_points(grid, h, True, pos, sig, numax, cube, c, pts)
    assert np.max(np.abs(got - full[pts])) < 1e-13 * np.max(np.abs(full))


def test_integer_shift_and_axis_swap_symmetry():
    rng = np.random.default_rng(5)
    grid, h = (24, 24, 24), 0.25
    psi = rng.standard_normal((24, 24, 24, 2))
    X = np.array([[2.61, 3.13, 2.37]])
    sig = [0.7]
    numax, cube = 3, 16
    c0 = oracle.project(grid, h, True, psi, X, sig, numax, cube)
    # shift by (2, -3, 5) grid steps and roll psi along: identical coefficients
    s = np.array([2, -3, 5])
    psi_s = np.roll(psi, shift=(s[2], s[1], s[0]), axis=(0, 1, 2))
    c1 = oracle.project(grid, h, True, psi_s, X + s * h, sig, numax, cube)
    assert np.max(np.abs(c1 - c0)) < 1e-13 * np.max(np.abs(c0))
    # swap x <-> y in psi and X: coefficients with nx <-> ny exchanged
    psi_t = np.ascontiguousarray(np.transpose(psi, (0, 2, 1, 3)))
    Xt = X[:, [1, 0, 2]]
    c2 = oracle.project(grid, h, True, psi_t, Xt, sig, numax, cube)
    st = _enumerate(numax)
    perm = [st.index((b, a, cc)) for a, b, cc in st]
    assert np.max(np.abs(c2[:, perm] - c0)) < 1e-13 * np.max(np.abs(c0))


# --------------------------------------------------------------------------- 5. forces
def _energy_grad_setup():
    rng = np.random.default_rng(17)
    grid, h = (20, 20, 20), 0.2
    psi = rng.standard_normal((20, 20, 20, 3))
    pos = np.array([[1.537, 2.081, 1.733], [2.911, 0.623, 3.147]])
    sig = np.array([0.66, 0.81])
    numax, cube = 3, 14
    g = rng.standard_normal((2, oracle.nstates(numax), 3))
    return grid, h, psi, pos, sig, numax, cube, g


def test_forces_match_central_finite_difference():
    grid, h, psi, pos, sig, numax, cube, g = _energy_grad_setup()
    f = oracle.forces(grid, h, True, psi, pos, sig, numax, cube, g)
    step = 1e-4
    for a in range(2):
        for d in range(3):
            pp, pm = pos.copy(), pos.copy()
            pp[a, d] += step
            pm[a, d] -= step
            # the cube origin must not move within +-step (positions are seeded away from grid planes)
            assert math.floor(pp[a, d] / h) == math.floor(pm[a, d] / h)
            ep = np.sum(g * oracle.project(grid, h, True, psi, pp, sig, numax, cube))
            em = np.sum(g * oracle.project(grid, h, True, psi, pm, sig, numax, cube))
            fd = (ep - em) / (2 * step)
            assert abs(f[a, d] - fd) <= 1e-7 * max(1.0, abs(fd)), (a, d, f[a, d], fd)


def test_forces_match_ladder_identity():
    """d/du phi_n = (1/sigma)[sqrt(n/2) phi_{n-1} - sqrt((n+1)/2) phi_{n+1}] (textbook ladder
    relation of Hermite functions), so dc/dX follows exactly from a projection at numax+1."""
    grid, h, psi, pos, sig, numax, cube, g = _energy_grad_setup()
    f = oracle.forces(grid, h, True, psi, pos, sig, numax, cube, g)
    cp = oracle.project(grid, h, True, psi, pos, sig, numax + 1, cube)
    big = _enumerate(numax + 1)
    ref = np.zeros((2, 3))
    for a in range(2):
        for k, m in enumerate(_enumerate(numax)):
            for d in range(3):
                dn = list(m)
                up = list(m)
                up[d] += 1
                term = math.sqrt((m[d] + 1) / 2) * cp[a, big.index(tuple(up))]
                if m[d] > 0:
                    dn[d] -= 1
                    term = term - math.sqrt(m[d] / 2) * cp[a, big.index(tuple(dn))]
                ref[a, d] += np.sum(g[a, k] * term) / sig[a]
    assert np.max(np.abs(f - ref)) < 1e-12 * np.max(np.abs(ref))


# --------------------------------------------------------------------------- spherical support (Sec. 6)
def test_sphere_brute_force_tiny():
    """Projection over the points of the cube inside a sphere of radius R (the paper's projection spheres)
    against the direct definition with scipy functions, periodic and clipped, R cutting through the cube."""
    rng = np.random.default_rng(17)
    grid, h, numax, cube = (10, 12, 11), 0.3, 2, 8
    pos = np.array([[1.31, 1.72, 1.55], [0.2, 3.1, 2.9]])
    sig = np.array([0.7, 0.9])
    psi = rng.standard_normal((grid[2], grid[1], grid[0], 2))
    for periodic in (True, False):
        for R in (0.65, 0.9, 1.07):
            got = oracle.project(grid, h, periodic, psi, pos, sig, numax, cube, rprj=R)
            ref = _brute_project(grid, h, periodic, psi, pos, sig, numax, cube, rprj=R)
            assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref)), (periodic, R)


def test_sphere_enclosing_the_cube_is_the_cube():
    rng = np.random.default_rng(18)
    grid, h, numax, cube = (16, 16, 16), 0.25, 3, 12
    pos = np.array([[2.1, 1.9, 2.3]])
    psi = rng.standard_normal((16, 16, 16, 3))
    c = rng.standard_normal((1, oracle.nstates(numax), 3))
    R = cube * h  # longer than any offset inside the cube
    assert np.array_equal(oracle.project(grid, h, True, psi, pos, [0.8], numax, cube),
                          oracle.project(grid, h, True, psi, pos, [0.8], numax, cube, rprj=R))
    assert np.array_equal(oracle.add(grid, h, True, psi, pos, [0.8], numax, cube, c),
                          oracle.add(grid, h, True, psi, pos, [0.8], numax, cube, c, rprj=R))


def test_sphere_equals_cube_of_masked_psi_and_adjoint():
    """Masking the support equals zeroing psi outside the sphere (one atom), and E stays the h^3-adjoint
    of P with the same support; expand_points agrees with add."""
    rng = np.random.default_rng(19)
    grid, h, numax, cube, R = (14, 14, 14), 0.25, 3, 12, 1.1
    X = np.array([[1.63, 1.77, 1.52]])
    sig = [0.75]
    psi = rng.standard_normal((14, 14, 14, 2))
    o = np.floor(X[0] / h).astype(int) - cube // 2 + 1
    u = [(o[d] + np.arange(cube)) * h - X[0, d] for d in range(3)]
    masked = np.zeros_like(psi)
    for iz in range(cube):
        for iy in range(cube):
            for ix in range(cube):
                if (u[0][ix] * u[0][ix] + u[1][iy] * u[1][iy]) + u[2][iz] * u[2][iz] <= R * R:
                    j = ((o[2] + iz) % 14, (o[1] + iy) % 14, (o[0] + ix) % 14)
                    masked[j] = psi[j]
    a = oracle.project(grid, h, True, psi, X, sig, numax, cube, rprj=R)
    b = oracle.project(grid, h, True, masked, X, sig, numax, cube)
    assert np.max(np.abs(a - b)) <= 1e-14 * np.max(np.abs(b))
    c = rng.standard_normal(a.shape)
    e = oracle.add(grid, h, True, np.zeros_like(psi), X, sig, numax, cube, c, rprj=R)
    lhs, rhs = float((a * c).sum()), h ** 3 * float((psi * e).sum())
    assert abs(lhs - rhs) <= 1e-13 * abs(lhs)
    pts = np.array([0, 500, 1234, 2000, 2743])
    ep = oracle.expand_points(grid, h, True, X, sig, numax, cube, c, pts, rprj=R)
    assert np.max(np.abs(ep - e.reshape(-1, 2)[pts])) <= 1e-14 * max(1.0, np.max(np.abs(e)))


def test_sphere_forces_match_finite_difference():
    """With no cube point near the sphere's surface the support does not change under a small shift, and
    the forces are the central differences of E = sum D c^2."""
    rng = np.random.default_rng(20)
    grid, h, numax, cube = (16, 16, 16), 0.25, 3, 12
    X = np.array([[2.03, 1.96, 2.11]])
    sig = [0.7]
    o = np.floor(X[0] / h).astype(int) - cube // 2 + 1
    u = [(o[d] + np.arange(cube)) * h - X[0, d] for d in range(3)]
    r = np.sqrt(u[0][None, None, :] ** 2 + u[1][None, :, None] ** 2 + u[2][:, None, None] ** 2).ravel()
    R = 0.5 * (np.sort(r)[200] + np.sort(r)[201])           # halfway between two point shells
    assert np.min(np.abs(r - R)) > 1e-3
    psi = rng.standard_normal((16, 16, 16, 2))
    Dm = rng.uniform(-1, 1, size=(1, oracle.nstates(numax)))
    c = oracle.project(grid, h, True, psi, X, sig, numax, cube, rprj=R)
    f = oracle.forces(grid, h, True, psi, X, sig, numax, cube, 2 * Dm[:, :, None] * c, rprj=R)
    step = 1e-5
    for d in range(3):
        e = []
        for sgn in (1, -1):
            Xs = X.copy()
            Xs[0, d] += sgn * step
            cs = oracle.project(grid, h, True, psi, Xs, sig, numax, cube, rprj=R)
            e.append(float((Dm[:, :, None] * cs * cs).sum()))
        fd = (e[0] - e[1]) / (2 * step)
        assert abs(f[0, d] - fd) <= 1e-7 * max(1.0, np.abs(f).max()), (d, f[0, d], fd)
