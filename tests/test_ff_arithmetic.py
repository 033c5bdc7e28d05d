"""The float-float dot step of the FP64-accurate form, emulated in exact rational arithmetic (CPU).

The step accumulates a*b for float pairs a = a.hi + a.lo, b = b.hi + b.lo into a running pair (s, c) with
p = fl(a.hi b.hi), TwoSum(s, p) = (t, (s - (t - bb)) + (p - bb)) with bb = t - s, and the product's exact
low part a.hi b.hi - p taken together with TwoSum's p - bb as one fused a.hi b.hi - bb (Ogita, Rump &
Oishi, Dot2, extended to pair inputs).  Checks: over 32-term dot products of random pairs the step is as
accurate as the textbook form with a separate error-free product (relative errors near 2^-48); if s + p
were fused into fma(a.hi, b.hi, s) -- a contraction the kernel prevents by computing p with __fmul_rn --
some inputs get errors of single-float size (about 1e-9 here).
"""
from fractions import Fraction as Fr

import numpy as np

f32 = np.float32


def _fma(a, b, c):
    """fma rounded once to float32, from the exact rational value."""
    return f32(float(Fr(float(a)) * Fr(float(b)) + Fr(float(c))))


def _step_textbook(s, c, ah, al, bh, bl):
    p = f32(ah * bh)
    e = _fma(ah, bh, -p)
    e = _fma(ah, bl, e)
    e = _fma(al, bh, e)
    t = f32(s + p)
    bb = f32(t - s)
    err = f32(f32(s - f32(t - bb)) + f32(p - bb))
    return t, f32(c + f32(err + e))


def _step_fused(s, c, ah, al, bh, bl, contract_sum=False):
    t = _fma(ah, bh, s) if contract_sum else f32(s + f32(ah * bh))
    bb = f32(t - s)
    q = _fma(ah, bh, -bb)
    q = _fma(ah, bl, q)
    q = _fma(al, bh, q)
    r = f32(s - f32(t - bb))
    return t, f32(c + f32(q + r))


def _dot(step, ah, al, bh, bl, **kw):
    s = c = f32(0)
    for i in range(len(ah)):
        s, c = step(s, c, ah[i], al[i], bh[i], bl[i], **kw)
    return Fr(float(s)) + Fr(float(c))


def _pairs(x):
    hi = x.astype(f32)
    lo = (x - hi.astype(np.float64)).astype(f32)
    return hi, lo


def test_fused_step_as_accurate_as_textbook_and_contraction_is_not():
    worst_contracted = 0.0
    for seed in range(8):
        rng = np.random.default_rng(7000 + seed)
        a = rng.standard_normal(32) * np.exp(rng.uniform(-3, 3, 32))
        b = rng.standard_normal(32)
        ah, al = _pairs(a)
        bh, bl = _pairs(b)
        exact = sum(Fr(float(ah[i])) * Fr(float(bh[i])) + Fr(float(ah[i])) * Fr(float(bl[i])) +
                    Fr(float(al[i])) * Fr(float(bh[i])) for i in range(32))
        scale = sum(abs(Fr(float(ah[i])) * Fr(float(bh[i]))) for i in range(32))  # sum of |leading products|

        def rel(v):
            return float(abs(v - exact) / scale)

        e_text = rel(_dot(_step_textbook, ah, al, bh, bl))
        e_fused = rel(_dot(_step_fused, ah, al, bh, bl))
        worst_contracted = max(worst_contracted, rel(_dot(_step_fused, ah, al, bh, bl, contract_sum=True)))
        assert e_text < 2.0 ** -44 and e_fused < 2.0 ** -44, (seed, e_text, e_fused)
        assert e_fused <= 4 * e_text + 2.0 ** -50, (seed, e_text, e_fused)
    # fusing s + p breaks TwoSum's exactness for some inputs: errors of single-float size
    assert worst_contracted > 2.0 ** -36, worst_contracted


def _split_model(v):
    """Bit-level model of the kernel's double -> (hi, lo) float split (integer instructions only)."""
    b = int(np.array(v, dtype=np.float64).view(np.uint64))
    lw, hw = b & 0xFFFFFFFF, b >> 32
    ax = hw & 0x7FFFFFFF
    ok = ((ax - 0x38100000) & 0xFFFFFFFF) < (0x47F00000 - 0x38100000)       # exponent in [897, 1150]
    hib = (((b >> 29) & 0xFFFFFFFF) - 0xC0000000) & 0xFFFFFFFF | (hw & 0x80000000)
    sb = ((hib - 0x1A000000) & 0xFFFFFFFF) & 0xFF800000
    hi = np.array(hib, dtype=np.uint32).view(np.float32) if ok else f32(0)
    lo = (f32(lw & 0x1FFFFFFF) * np.array(sb, dtype=np.uint32).view(np.float32)) if (ok and ax >= 0x3B500000) \
        else f32(0)
    return f32(hi), f32(lo)


def test_branch_free_split_of_a_double():
    """hi carries the sign, exponent and top 23 mantissa bits of v (truncation), lo the remainder rounded once
    to float: |v - (hi + lo)| <= 2^-48 |v| wherever lo is a normal float; values outside the float normal
    range give (0, 0); below 2^-74 lo is dropped (relative error below 2^-23)."""
    rng = np.random.default_rng(7100)
    vals = np.concatenate([rng.standard_normal(3000) * 10.0 ** rng.uniform(-37, 37, 3000),
                           [1.0, -1.0, 2.0 ** -126, -(2.0 ** -126), 2.0 ** 127 * 1.999, 2.0 ** -74, 2.0 ** -73]])
    for v in vals:
        hi, lo = _split_model(v)
        if not 2.0 ** -126 <= abs(v) < 2.0 ** 128:
            assert (hi, lo) == (0.0, 0.0), v
            continue
        assert np.float32(hi) == np.float32(np.float64(hi)), v
        assert abs(float(hi)) <= abs(v) and (hi == 0 or np.sign(hi) == np.sign(v)), v   # truncation toward zero
        err = abs(Fr(float(v)) - Fr(float(hi)) - Fr(float(lo)))
        bound = Fr(2) ** -48 if abs(v) >= 2.0 ** -73 else Fr(2) ** -23
        assert err <= bound * abs(Fr(float(v))), (v, float(err))
    for v in [0.0, -0.0, 2.0 ** -127, 1e-300, 2.0 ** 128, -1e300]:
        assert _split_model(v) == (0.0, 0.0), v
