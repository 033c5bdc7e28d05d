"""Shared helpers for the GPU parity tests."""
import numpy as np
import pytest

# FP64 bar: norm-wise relative error per atom, and max error relative to the largest reference value.
TOL_FP64 = 1e-12
# FP32 CUDA-core form against the oracle run on the same (storage-rounded) input: FP32 rounding of
# the function tables (2^-24) and of the three pass accumulations (~C terms each) bound the norm-wise
# error by a few 1e-7; 2e-6 leaves margin for the 32-term sums.
TOL_FP32 = 2e-6


def require_gpu():
    import torch
    if not torch.cuda.is_available():
        pytest.skip("needs a CUDA GPU")


def rel_norm(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.linalg.norm(ref)
    return np.linalg.norm(got - ref) / (den if den > 0 else 1.0)


def rel_max(got, ref):
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    den = np.max(np.abs(ref))
    return np.max(np.abs(got - ref)) / (den if den > 0 else 1.0)


def assert_coeff_close(got, ref, tol):
    """Per-atom norm-wise check plus a global max check."""
    got = np.asarray(got, dtype=np.float64)
    for a in range(ref.shape[0]):
        e = rel_norm(got[a], ref[a])
        assert e <= tol, f"atom {a}: norm-wise relative error {e:.3e} > {tol:.1e}"
    e = rel_max(got, ref)
    assert e <= tol, f"max relative error {e:.3e} > {tol:.1e}"
