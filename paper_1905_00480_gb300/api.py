"""PyTorch-facing binding of libsho: same names as the C ABI, argument marshalling only.

PyTorch provides device memory and streams; every step of projection, expansion and forces runs in
the library's CUDA kernels.  Tensors must live on a CUDA device; there is no CPU path.

Layouts (see include/sho.h): psi [Nz][Ny][Nx][B] contiguous, coefficients [A][N][B], positions [A][3]
and sigma [A] (any device; they are copied to the host as the C ABI expects).
"""
from __future__ import annotations

import ctypes
import threading

import numpy as np
import torch

from . import _native as N

_TORCH_DT = {torch.float64: "f64", torch.float32: "f32", torch.bfloat16: "bf16"}


def nstates(numax: int) -> int:
    """(numax+1)(numax+2)(numax+3)/6 (eq. SHO_basis_size)."""
    return int(N.lib().sho_nstates(int(numax)))


def max_spacing(sigma: float, numax: int) -> float:
    """h_max = pi sigma / sqrt(2 numax + 1) (eq. max_grid_spacing)."""
    return float(N.lib().sho_max_spacing(float(sigma), int(numax)))


class Handle:
    """Owns a libsho handle (device workspace, call ordering) for one CUDA device."""

    def __init__(self, device: int = 0, strict: bool = False):
        self._h = ctypes.c_void_p()
        self.device = int(device)
        N.check(N.lib().sho_create(ctypes.byref(self._h), self.device), "sho_create")
        if strict:
            N.check(N.lib().sho_set_strict(self._h, 1), "sho_set_strict")

    @property
    def ptr(self):
        return self._h

    def sync(self):
        N.check(N.lib().sho_sync(self._h), "sho_sync")

    def set_expand_kernel(self, kernel: str):
        """sho_set_expand_kernel: "auto", "mma_sync" or "tcgen05" x-pass of the TF32 / BF16 expansions
        ("tcgen05" also selects the digit-sliced tensor-core x-pass of the FF64 expansion)."""
        N.check(N.lib().sho_set_expand_kernel(self._h, {"auto": 0, "mma_sync": 1, "tcgen05": 2}[kernel]),
                "sho_set_expand_kernel")

    def set_project_kernel(self, kernel: str):
        """sho_set_project_kernel: "auto" / "mma_sync" (the float-float CUDA-core kernel of the FF64
        projection) or "tcgen05" (its digit-sliced tensor-core x-pass, where it applies)."""
        N.check(N.lib().sho_set_project_kernel(self._h, {"auto": 0, "mma_sync": 1, "tcgen05": 2}[kernel]),
                "sho_set_project_kernel")

    def set_device_checks(self, on: bool = True):
        """sho_set_device_checks: the FP64 / FF64 kernels check every psi, coefficient and intermediate index."""
        N.check(N.lib().sho_set_device_checks(self._h, 1 if on else 0), "sho_set_device_checks")

    def set_support_radius(self, rprj: float):
        """sho_set_support_radius: spherical projector support of radius rprj (0 = the whole cube)."""
        N.check(N.lib().sho_set_support_radius(self._h, float(rprj)), "sho_set_support_radius")

    def close(self):
        if self._h:
            N.lib().sho_destroy(self._h)
            self._h = ctypes.c_void_p()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


_handles = {}
_hlock = threading.Lock()


def default_handle(device: int) -> Handle:
    with _hlock:
        h = _handles.get(device)
        if h is None:
            h = _handles[device] = Handle(device)
        return h


def _grid(psi: torch.Tensor, h: float, periodic: bool) -> N.sho_grid:
    g = N.sho_grid()
    nz, ny, nx = psi.shape[0], psi.shape[1], psi.shape[2]
    g.n[0], g.n[1], g.n[2] = int(nx), int(ny), int(nz)
    g.h = float(h)
    g.periodic = 1 if periodic else 0
    return g


def _host_f64(x, shape_last=None):
    if isinstance(x, torch.Tensor):
        x = x.detach().to("cpu", torch.float64).numpy()
    a = np.ascontiguousarray(np.asarray(x, dtype=np.float64))
    if shape_last is not None:
        a = a.reshape(-1, shape_last)
    return a


def _dp(a: np.ndarray):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double))


def _check_psi(psi: torch.Tensor):
    if not psi.is_cuda:
        raise ValueError("psi must be a CUDA tensor (there is no CPU path)")
    if psi.dim() != 4 or not psi.is_contiguous():
        raise ValueError("psi must be a contiguous [Nz][Ny][Nx][B] tensor")
    if psi.dtype not in _TORCH_DT:
        raise ValueError(f"unsupported psi dtype {psi.dtype}")


def _stream_ptr(psi: torch.Tensor, stream):
    s = stream if stream is not None else torch.cuda.current_stream(psi.device)
    return ctypes.c_void_p(s.cuda_stream)


def _coeff_dtype(prec: str):
    return torch.float64 if prec in ("fp64", "ff64") else torch.float32


def project(psi: torch.Tensor, pos, sigma, numax: int, cube: int, h: float, periodic: bool = True,
            prec: str = "fp64", out: torch.Tensor = None, handle: Handle = None, stream=None) -> torch.Tensor:
    """sho_project: c[a][k][b] = h^3 sum over the atom's cube of Psi_k(u) psi[j][b]."""
    _check_psi(psi)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A, B = pos_h.shape[0], psi.shape[3]
    cdt = _coeff_dtype(prec)
    if out is None:
        out = torch.empty((A, nstates(numax), B), dtype=cdt, device=psi.device)
    elif out.dtype != cdt or not out.is_contiguous() or tuple(out.shape) != (A, nstates(numax), B):
        raise ValueError("out has the wrong dtype, shape or layout")
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid(psi, h, periodic)
    st = N.lib().sho_project(hd.ptr, ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()), N.DTYPES[_TORCH_DT[psi.dtype]],
                             B, A, _dp(pos_h), _dp(sig_h), int(numax), int(cube), N.PRECS[prec],
                             ctypes.c_void_p(out.data_ptr()), N.DTYPES[_TORCH_DT[cdt]], _stream_ptr(psi, stream))
    N.check(st, "sho_project" if st != N.SHO_ERR_CUDA else
            f"sho_project ({N.lib().sho_last_cuda_error(hd.ptr).decode()})")
    return out


def project_path(psi: torch.Tensor, numax: int, cube: int, h: float, periodic: bool = True, prec: str = "fp64") -> str:
    """sho_project_path: "plane" (plane sweep) or "atom" (per-atom kernels) for a projection of psi."""
    _check_psi(psi)
    g = _grid(psi, h, periodic)
    cdt = _coeff_dtype(prec)
    r = N.lib().sho_project_path(ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()), N.DTYPES[_TORCH_DT[psi.dtype]],
                                 psi.shape[3], int(numax), int(cube), N.PRECS[prec], N.DTYPES[_TORCH_DT[cdt]])
    if r < 0:
        N.check(r, "sho_project_path")
    return {1: "atom", 2: "plane"}[r]


def _grid_complex(psi: torch.Tensor, h: float):
    g = N.sho_grid()
    g.n[0], g.n[1], g.n[2] = int(psi.shape[2]), int(psi.shape[1]), int(psi.shape[0])
    g.h, g.periodic = float(h), 1
    return g


def _check_complex(t: torch.Tensor, what: str, dims: int, prec: str = "fp64"):
    want = torch.complex64 if prec == "fp32" else torch.complex128
    if not t.is_cuda or not t.is_contiguous() or t.dtype != want or t.dim() != dims:
        raise ValueError(f"{what} must be a contiguous CUDA {str(want)[6:]} tensor with {dims} dimensions "
                         f"for prec {prec!r}")


def project_bloch(psi: torch.Tensor, kvec, pos, sigma, numax: int, cube: int, h: float, out: torch.Tensor = None,
                  handle: Handle = None, stream=None, prec: str = "fp64") -> torch.Tensor:
    """sho_project_bloch: complex Bloch psi [Nz][Ny][Nx][B] (periodic grid) -> complex [A][N][B].
    prec "fp64" (complex FMAs on the FP64 pipe) or "ff64" (float-float passes, FP64-accurate), both on
    complex128 data, or "fp32" (the FP32 CUDA-core kernels) on complex64 data."""
    _check_complex(psi, "psi", 4, prec)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    k = _host_f64(kvec).reshape(3)
    A, B = pos_h.shape[0], psi.shape[3]
    if out is None:
        out = torch.empty((A, nstates(numax), B), dtype=psi.dtype, device=psi.device)
    _check_complex(out, "out", 3, prec)
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid_complex(psi, h)
    st = N.lib().sho_project_bloch(hd.ptr, ctypes.byref(g), _dp(k), ctypes.c_void_p(psi.data_ptr()), B, A,
                                   _dp(pos_h), _dp(sig_h), int(numax), int(cube), N.PRECS[prec],
                                   ctypes.c_void_p(out.data_ptr()), _stream_ptr(psi, stream))
    N.check(st, "sho_project_bloch")
    return out


def add_bloch(psi: torch.Tensor, coeff: torch.Tensor, kvec, pos, sigma, numax: int, cube: int, h: float,
              handle: Handle = None, stream=None, prec: str = "fp64") -> torch.Tensor:
    """sho_add_bloch (in place): psi += sum_a sum_k c Psi_k e^{-i k.T} for complex Bloch psi.
    prec "fp64", "ff64" or "fp32" as for project_bloch."""
    _check_complex(psi, "psi", 4, prec)
    _check_complex(coeff, "coeff", 3, prec)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    k = _host_f64(kvec).reshape(3)
    A, B = pos_h.shape[0], psi.shape[3]
    if tuple(coeff.shape) != (A, nstates(numax), B):
        raise ValueError("coeff must be [A][N][B]")
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid_complex(psi, h)
    st = N.lib().sho_add_bloch(hd.ptr, ctypes.byref(g), _dp(k), ctypes.c_void_p(coeff.data_ptr()), B, A, _dp(pos_h),
                               _dp(sig_h), int(numax), int(cube), N.PRECS[prec], ctypes.c_void_p(psi.data_ptr()),
                               _stream_ptr(psi, stream))
    N.check(st, "sho_add_bloch")
    return psi


def radial_labels(numax: int):
    """sho_radial_labels: (nr, l, m) of the radial SHO states in the library's order."""
    n = nstates(numax)
    nr, ell, m = ((ctypes.c_int * n)() for _ in range(3))
    N.check(N.lib().sho_radial_labels(int(numax), nr, ell, m), "sho_radial_labels")
    return [(nr[i], ell[i], m[i]) for i in range(n)]


def radial_matrix(numax: int):
    """sho_radial_matrix: U[k][j] = <Psi_j^rad | Psi_k^cart> as a float64 numpy array [N][N]."""
    import numpy as np
    n = nstates(numax)
    U = np.zeros((n, n), dtype=np.float64)
    N.check(N.lib().sho_radial_matrix(int(numax), U.ctypes.data_as(ctypes.POINTER(ctypes.c_double))),
            "sho_radial_matrix")
    return U


def to_radial(coeff: torch.Tensor, numax: int, inverse: bool = False, out: torch.Tensor = None,
              handle: Handle = None, stream=None) -> torch.Tensor:
    """sho_radial_transform: Cartesian [A][N][B] coefficients to radial ones (inverse=True: back)."""
    if not coeff.is_cuda or not coeff.is_contiguous() or coeff.dim() != 3 or coeff.shape[1] != nstates(numax):
        raise ValueError("coeff must be a contiguous CUDA tensor [A][N][B]")
    if coeff.dtype not in (torch.float64, torch.float32):
        raise ValueError("coeff must be float64 or float32")
    if out is None:
        out = torch.empty_like(coeff)
    elif out.shape != coeff.shape or out.dtype != coeff.dtype or not out.is_contiguous():
        raise ValueError("out has the wrong dtype, shape or layout")
    hd = handle or default_handle(coeff.device.index or 0)
    A, _, B = coeff.shape
    st = N.lib().sho_radial_transform(hd.ptr, A, int(numax), B, ctypes.c_void_p(coeff.data_ptr()),
                                      ctypes.c_void_p(out.data_ptr()), N.DTYPES[_TORCH_DT[coeff.dtype]],
                                      1 if inverse else 0, _stream_ptr(coeff, stream))
    N.check(st, "sho_radial_transform")
    return out


def add(psi: torch.Tensor, coeff: torch.Tensor, pos, sigma, numax: int, cube: int, h: float, periodic: bool = True,
        prec: str = "fp64", handle: Handle = None, stream=None, alpha: float = 1.0,
        overwrite: bool = False) -> torch.Tensor:
    """sho_add (in place): psi[j][b] += sum_a sum_k c[a][k][b] Psi_k(u).  Returns psi.

    With alpha != 1 or overwrite=True it is sho_add_scaled: psi = (0 if overwrite else psi) + alpha E c,
    the factor applied inside the kernels and the clearing done by the library."""
    _check_psi(psi)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A, B = pos_h.shape[0], psi.shape[3]
    if not coeff.is_cuda or not coeff.is_contiguous() or tuple(coeff.shape) != (A, nstates(numax), B):
        raise ValueError("coeff must be a contiguous CUDA tensor [A][N][B]")
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid(psi, h, periodic)
    tail = (ctypes.c_void_p(coeff.data_ptr()), N.DTYPES[_TORCH_DT[coeff.dtype]], B, A, _dp(pos_h), _dp(sig_h),
            int(numax), int(cube), N.PRECS[prec], ctypes.c_void_p(psi.data_ptr()), N.DTYPES[_TORCH_DT[psi.dtype]],
            _stream_ptr(psi, stream))
    if alpha == 1.0 and not overwrite:
        name = "sho_add"
        st = N.lib().sho_add(hd.ptr, ctypes.byref(g), *tail)
    else:
        name = "sho_add_scaled"
        st = N.lib().sho_add_scaled(hd.ptr, ctypes.byref(g), float(alpha), 1 if overwrite else 0, *tail)
    N.check(st, name if st != N.SHO_ERR_CUDA else f"{name} ({N.lib().sho_last_cuda_error(hd.ptr).decode()})")
    return psi


def forces(psi: torch.Tensor, dEdc: torch.Tensor, pos, sigma, numax: int, cube: int, h: float,
           periodic: bool = True, prec: str = "fp64", out: torch.Tensor = None, handle: Handle = None,
           stream=None) -> torch.Tensor:
    """sho_forces: dEdX[a][d] = sum_{k,b} dEdc[a][k][b] d c[a][k][b] / d X[a][d] (FP64 result)."""
    _check_psi(psi)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A, B = pos_h.shape[0], psi.shape[3]
    if not dEdc.is_cuda or not dEdc.is_contiguous() or tuple(dEdc.shape) != (A, nstates(numax), B):
        raise ValueError("dEdc must be a contiguous CUDA tensor [A][N][B]")
    if out is None:
        out = torch.empty((A, 3), dtype=torch.float64, device=psi.device)
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid(psi, h, periodic)
    st = N.lib().sho_forces(hd.ptr, ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()),
                            N.DTYPES[_TORCH_DT[psi.dtype]], B, A, _dp(pos_h), _dp(sig_h), int(numax), int(cube),
                            N.PRECS[prec], ctypes.c_void_p(dEdc.data_ptr()), N.DTYPES[_TORCH_DT[dEdc.dtype]],
                            ctypes.cast(ctypes.c_void_p(out.data_ptr()), ctypes.POINTER(ctypes.c_double)),
                            _stream_ptr(psi, stream))
    N.check(st, "sho_forces")
    return out


def apply_nonlocal(psi: torch.Tensor, hpsi: torch.Tensor, D: torch.Tensor, pos, sigma, numax: int, cube: int,
                   h: float, periodic: bool = True, prec: str = "fp64", handle: Handle = None,
                   stream=None) -> torch.Tensor:
    """sho_apply_nonlocal (in place on hpsi): hpsi += sum_a |k> D[a][k][k'] <k'|psi>."""
    _check_psi(psi)
    _check_psi(hpsi)
    if hpsi.shape != psi.shape or hpsi.dtype != psi.dtype:
        raise ValueError("hpsi must match psi in shape and dtype")
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A, B = pos_h.shape[0], psi.shape[3]
    Ns = nstates(numax)
    if not D.is_cuda or not D.is_contiguous() or tuple(D.shape) != (A, Ns, Ns) or D.dtype != _coeff_dtype(prec):
        raise ValueError("D must be a contiguous CUDA tensor [A][N][N] of the form's coefficient dtype")
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid(psi, h, periodic)
    st = N.lib().sho_apply_nonlocal(hd.ptr, ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()),
                                    N.DTYPES[_TORCH_DT[psi.dtype]], B, A, _dp(pos_h), _dp(sig_h), int(numax),
                                    int(cube), N.PRECS[prec], ctypes.c_void_p(D.data_ptr()),
                                    ctypes.c_void_p(hpsi.data_ptr()), _stream_ptr(psi, stream))
    N.check(st, "sho_apply_nonlocal")
    return hpsi


# ------------------------------------------------------------------------ stored-projector baseline
def usu_build(pos, sigma, numax: int, cube: int, grid_shape, h: float, periodic: bool = True, device=0,
              handle: Handle = None, stream=None, nproj: int = None, dtype=torch.float64) -> torch.Tensor:
    """sho_usu_build: sample every atom's first nproj projector values (default: all states of numax)
    onto its cube, [A][C^3][nproj] of dtype (float64 or float32) on the device."""
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A = pos_h.shape[0]
    nproj = nstates(numax) if nproj is None else int(nproj)
    if dtype not in (torch.float64, torch.float32):
        raise ValueError("stored projectors are float64 or float32")
    dev = torch.device("cuda", device) if isinstance(device, int) else torch.device(device)
    proj = torch.empty((A, cube ** 3, nproj), dtype=dtype, device=dev)
    hd = handle or default_handle(dev.index or 0)
    g = N.sho_grid()
    g.n[0], g.n[1], g.n[2] = int(grid_shape[0]), int(grid_shape[1]), int(grid_shape[2])
    g.h, g.periodic = float(h), 1 if periodic else 0
    s = stream if stream is not None else torch.cuda.current_stream(dev)
    st = N.lib().sho_usu_build(hd.ptr, ctypes.byref(g), A, _dp(pos_h), _dp(sig_h), int(numax), nproj, int(cube),
                               N.DTYPES[_TORCH_DT[dtype]], ctypes.c_void_p(proj.data_ptr()),
                               ctypes.c_void_p(s.cuda_stream))
    N.check(st, "sho_usu_build")
    return proj


def usu_project(psi: torch.Tensor, proj: torch.Tensor, pos, sigma, numax: int, cube: int, h: float,
                periodic: bool = True, out: torch.Tensor = None, handle: Handle = None, stream=None):
    """sho_usu_project: the projection with stored projector values (psi, proj and the result share one
    dtype, float64 or float32); the projector count is proj.shape[2] (numax is accepted for symmetry with
    usu_build and ignored)."""
    _check_psi(psi)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A, B = pos_h.shape[0], psi.shape[3]
    nproj = int(proj.shape[2])
    if psi.dtype != proj.dtype or psi.dtype not in (torch.float64, torch.float32):
        raise ValueError("psi and proj must both be float64 or both float32")
    if out is None:
        out = torch.empty((A, nproj, B), dtype=psi.dtype, device=psi.device)
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid(psi, h, periodic)
    st = N.lib().sho_usu_project(hd.ptr, ctypes.byref(g), ctypes.c_void_p(psi.data_ptr()), B, A, _dp(pos_h),
                                 _dp(sig_h), nproj, int(cube), N.DTYPES[_TORCH_DT[psi.dtype]],
                                 ctypes.c_void_p(proj.data_ptr()),
                                 ctypes.c_void_p(out.data_ptr()), _stream_ptr(psi, stream))
    N.check(st, "sho_usu_project")
    return out


def usu_add(psi: torch.Tensor, coeff: torch.Tensor, proj: torch.Tensor, pos, sigma, numax: int, cube: int, h: float,
            periodic: bool = True, handle: Handle = None, stream=None):
    """sho_usu_add (in place): the expansion with stored projector values (psi, coeff and proj share one
    dtype, float64 or float32)."""
    _check_psi(psi)
    pos_h = _host_f64(pos, 3)
    sig_h = _host_f64(sigma).reshape(-1)
    A, B = pos_h.shape[0], psi.shape[3]
    if tuple(coeff.shape) != (A, int(proj.shape[2]), B) or coeff.dtype != psi.dtype or proj.dtype != psi.dtype:
        raise ValueError(f"coeff must be {psi.dtype} [{A}][{int(proj.shape[2])}][{B}] like psi and proj, "
                         f"got {coeff.dtype} {tuple(coeff.shape)}")
    hd = handle or default_handle(psi.device.index or 0)
    g = _grid(psi, h, periodic)
    st = N.lib().sho_usu_add(hd.ptr, ctypes.byref(g), ctypes.c_void_p(coeff.data_ptr()), B, A, _dp(pos_h),
                             _dp(sig_h), int(proj.shape[2]), int(cube), N.DTYPES[_TORCH_DT[psi.dtype]],
                             ctypes.c_void_p(proj.data_ptr()),
                             ctypes.c_void_p(psi.data_ptr()), _stream_ptr(psi, stream))
    N.check(st, "sho_usu_add")
    return psi
