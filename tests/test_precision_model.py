"""Where the tolerances of the reduced-precision forms come from (CPU).

The x-pass of each form is emulated in numpy with the form's operand rounding, products of rounded
operands (exact in FP32) and FP32 accumulation; the y- and z-passes run in FP32, as on the GPU.  The
emulation is compared with the FP64 oracle on the same FP32 psi.  Each form's error must land inside the
tolerance the GPU parity tests use (TF32 2e-3, 3xTF32 1e-5, BF16 1.5e-2, split-FP16 1e-5) and near the
value the operand rounding predicts: about 2u for one rounded operand pair (u = 2^-11 TF32, 2^-8 BF16),
about 2^-22 for the split forms, whose correction products restore the operands to 22 bits.

Rounding as the kernels apply it: TF32 by cvt.rna (nearest, ties away from zero, 10 mantissa bits); BF16
and FP16 by round-to-nearest-even; 3xTF32 a*b ~ hi_a hi_b + hi_a lo_b + lo_a hi_b with hi = tf32(x),
lo = tf32(x - hi); split-FP16 the same with hi = fp16(x), lo = fp16((x - hi) 2^11) 2^-11.
"""
import numpy as np
import pytest

import oracle

TOL = {"fp32": 1e-5, "tf32": 2e-3, "3xtf32": 1e-5, "bf16": 1.5e-2, "split_fp16": 1e-5}
# what the operand rounding predicts for the norm-wise error (order of magnitude: [low, high])
EXPECT = {"fp32": (1e-9, 2e-6), "tf32": (5e-5, 2e-3), "3xtf32": (1e-9, 2e-6), "bf16": (5e-4, 1.5e-2),
          "split_fp16": (1e-9, 2e-6)}


def _tf32(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x1000) & 0xFFFFE000).astype(np.uint32)   # magnitude + half ulp, truncate: ties away
    return b.view(np.float32)


def _bf16(x):
    b = np.asarray(x, dtype=np.float32).view(np.uint32).astype(np.uint64)
    b = ((b + 0x7FFF + ((b >> 16) & 1)) & 0xFFFF0000).astype(np.uint32)   # nearest even
    return b.view(np.float32)


def _fp16(x):
    return np.asarray(x, dtype=np.float32).astype(np.float16).astype(np.float32)


def _xpass(psi, tx, mode):
    """T1[z][y][n][b] = sum_x psi[z][y][x][b] tx[x][n] with the form's operands and FP32 sums."""
    def mm(a, b):  # FP32 products of FP32-exact operands, FP32 accumulation
        return np.einsum("zyxb,xn->zynb", a.astype(np.float32), b.astype(np.float32), dtype=np.float32)
    if mode == "fp32":
        return mm(psi, tx)
    if mode == "tf32":
        return mm(_tf32(psi), _tf32(tx))
    if mode == "bf16":
        return mm(_bf16(psi), _bf16(tx))
    if mode == "3xtf32":
        ah, bh = _tf32(psi), _tf32(tx)
        al, bl = _tf32(psi - ah), _tf32(tx - bh)
        return mm(ah, bh) + (mm(ah, bl) + mm(al, bh))
    ah, bh = _fp16(psi), _fp16(tx)
    al, bl = _fp16((psi - ah) * 2048.0), _fp16((tx - bh) * 2048.0)
    return mm(ah, bh) + np.float32(1.0 / 2048.0) * (mm(ah, bl) + mm(al, bh))


def _tables(X, sigma, numax, cube, h):
    """phi_n at the cube offsets u = (o + i) h - X per axis (FP64, rounded to FP32 as the GPU stores them)."""
    out = []
    for d in range(3):
        o = int(np.floor(X[d] / h)) - cube // 2 + 1
        t = np.array([[oracle.phi(n, (o + i) * h - X[d], sigma) for n in range(numax + 1)] for i in range(cube)])
        out.append(t.astype(np.float32))
    return out


@pytest.mark.parametrize("mode", sorted(TOL))
def test_emulated_form_error_fits_its_tolerance(mode):
    rng = np.random.default_rng(5150)
    numax, cube, h, sigma, B = 5, 16, 0.25, 0.8, 24
    grid = (cube, cube, cube)
    X = np.array([7.37, 7.52, 7.18]) * h    # the cube is the grid: o = 0 on every axis
    psi = rng.standard_normal((cube, cube, cube, B)).astype(np.float32)
    tx, ty, tz = _tables(X, sigma, numax, cube, h)
    t1 = _xpass(psi, tx, mode)                                              # [z][y][nx][b]
    t2 = np.einsum("zynb,ym->zmnb", t1, ty, dtype=np.float32)               # [z][ny][nx][b]
    c3 = np.einsum("zmnb,zk->kmnb", t2, tz, dtype=np.float32) * np.float32(h ** 3)  # [nz][ny][nx][b]
    states = oracle.basis(numax)
    got = np.stack([c3[nz, ny, nx] for nx, ny, nz in states])[None]         # [1][N][B]
    ref = oracle.project(grid, h, False, psi.astype(np.float64), X[None], [sigma], numax, cube)
    err = np.linalg.norm(got - ref) / np.linalg.norm(ref)
    lo, hi = EXPECT[mode]
    assert err <= TOL[mode], (mode, err)
    assert lo <= err <= hi, (mode, err)
