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
