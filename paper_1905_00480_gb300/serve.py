"""Python binding of the serving loop (sho_server_* in include/sho.h): argument marshalling only.

The scheduler, admission by memory budget, slot streams and latency records are native (libsho);
this class wraps the handle and converts tensors to pointers.
"""
from __future__ import annotations

import ctypes

import numpy as np
import torch

from . import _native as N
from .api import _host_f64, _dp, _TORCH_DT, nstates

OPS = {"project": 0, "expand": 1}


class Server:
    def __init__(self, device: int = 0, budget_bytes: int = 64 << 30, slots: int = 4):
        self._s = ctypes.c_void_p()
        self.device = device
        N.check(N.lib().sho_server_create(ctypes.byref(self._s), int(device), int(budget_bytes), int(slots)),
                "sho_server_create")
        self._meta = {}

    def close(self):
        if self._s:
            N.lib().sho_server_destroy(self._s)
            self._s = ctypes.c_void_p()

    def __enter__(self):
        return self

    def __exit__(self, *exc):
        self.close()

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def register(self, psi: torch.Tensor, pos, sigma, numax: int, cube: int, h: float, periodic: bool = True) -> int:
        """Copy psi ([Nz][Ny][Nx][B], host or device) into server-owned device memory; returns the id."""
        if psi.dim() != 4 or not psi.is_contiguous():
            raise ValueError("psi must be a contiguous [Nz][Ny][Nx][B] tensor")
        g = N.sho_grid()
        g.n[0], g.n[1], g.n[2] = int(psi.shape[2]), int(psi.shape[1]), int(psi.shape[0])
        g.h, g.periodic = float(h), 1 if periodic else 0
        pos_h = _host_f64(pos, 3)
        sig_h = _host_f64(sigma).reshape(-1)
        sid = ctypes.c_int()
        st = N.lib().sho_system_register(self._s, ctypes.byref(g), int(psi.shape[3]), pos_h.shape[0], _dp(pos_h),
                                         _dp(sig_h), int(numax), int(cube), N.DTYPES[_TORCH_DT[psi.dtype]],
                                         ctypes.c_void_p(psi.data_ptr()), ctypes.byref(sid))
        N.check(st, "sho_system_register")
        cdt = torch.float64 if psi.dtype == torch.float64 else torch.float32
        self._meta[sid.value] = (tuple(psi.shape), psi.dtype, (pos_h.shape[0], nstates(numax), int(psi.shape[3])), cdt)
        return sid.value

    def unregister(self, sid: int):
        N.check(N.lib().sho_system_unregister(self._s, int(sid)), "sho_system_unregister")
        self._meta.pop(sid, None)

    def read(self, sid: int, psi: bool = True, coeff: bool = True):
        shape, dt, cshape, cdt = self._meta[sid]
        p = torch.empty(shape, dtype=dt) if psi else None
        c = torch.empty(cshape, dtype=cdt) if coeff else None
        st = N.lib().sho_system_read(self._s, int(sid), ctypes.c_void_p(p.data_ptr()) if p is not None else None,
                                     ctypes.c_void_p(c.data_ptr()) if c is not None else None)
        N.check(st, "sho_system_read")
        return p, c

    def write_coeff(self, sid: int, coeff: torch.Tensor):
        shape, dt, cshape, cdt = self._meta[sid]
        if tuple(coeff.shape) != cshape or coeff.dtype != cdt or not coeff.is_contiguous():
            raise ValueError("coefficients have the wrong shape, dtype or layout")
        N.check(N.lib().sho_system_write_coeff(self._s, int(sid), ctypes.c_void_p(coeff.data_ptr())),
                "sho_system_write_coeff")

    def submit(self, sid: int, op: str, prec: str = "fp32") -> int:
        t = ctypes.c_uint64()
        N.check(N.lib().sho_submit(self._s, int(sid), OPS[op], N.PRECS[prec], ctypes.byref(t)), "sho_submit")
        return t.value

    def wait(self, ticket: int, timeout_ms: int = 60000, with_latency: bool = False):
        """sho_wait_status: returns the request's status (0 = ok), or (status, latency_ms) with
        with_latency=True; raises TimeoutError when the request is not complete within timeout_ms (the
        ticket stays valid)."""
        rs = ctypes.c_int()
        lat = ctypes.c_double()
        st = N.lib().sho_wait_status(self._s, ctypes.c_uint64(ticket), int(timeout_ms), ctypes.byref(rs),
                                     ctypes.byref(lat))
        if st == -8:
            raise TimeoutError(f"ticket {ticket} not complete after {timeout_ms} ms")
        N.check(st, "sho_wait_status")
        return (rs.value, lat.value) if with_latency else rs.value

    def cancel(self, ticket: int) -> int:
        """sho_cancel: 0 when the queued request was removed, SHO_ERR_STATE (-11) when it already started
        or finished."""
        return int(N.lib().sho_cancel(self._s, ctypes.c_uint64(ticket)))

    def fault_hold(self, sid: int, hold: bool = True):
        """sho_fault_hold (fault injection): while held, a running request of the system is not retired."""
        N.check(N.lib().sho_fault_hold(self._s, int(sid), 1 if hold else 0), "sho_fault_hold")

    def fault_pipeline(self, cycles: int = 0, rows: int = -1):
        """sho_fault_server_pipeline (fault injection): wait limit and producer row stop of every slot."""
        N.check(N.lib().sho_fault_server_pipeline(self._s, int(cycles), int(rows)), "sho_fault_server_pipeline")

    def stats(self) -> dict:
        s = N.sho_server_stats()
        N.check(N.lib().sho_server_get_stats(self._s, ctypes.byref(s)), "sho_server_get_stats")
        return {f: getattr(s, f) for f, _ in s._fields_}

    def reset_stats(self):
        N.check(N.lib().sho_server_reset_stats(self._s), "sho_server_reset_stats")
