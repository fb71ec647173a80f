"""Thin Python binding of the C ABI (include/sipstokes.h).

Marshalling only: each method forwards torch CUDA tensors (device
pointers) and the current CUDA stream to the entry point of the same name,
and raises ``SipError`` with the library's message on a non-OK status.
Every step of the computation runs in the CUDA library.
"""
import ctypes

import numpy as np
import torch

from . import _lib
from ._lib import SipError, ProblemDesc, SolveOpts, SolveReport, BC, PREC


def _ptr(t, dtype):
    if t is None:
        return None
    if not isinstance(t, torch.Tensor) or not t.is_cuda:
        raise TypeError("expected a CUDA tensor")
    if t.dtype != dtype:
        raise TypeError(f"expected {dtype}, got {t.dtype}")
    if not t.is_contiguous():
        raise ValueError("tensor must be contiguous")
    return ctypes.c_void_p(t.data_ptr())


def _stream(stream):
    s = stream if stream is not None else torch.cuda.current_stream()
    return ctypes.c_void_p(s.cuda_stream)


class Context:
    """sip_ctx: the library context on one CUDA device."""

    def __init__(self, device=0):
        self.lib = _lib.load()
        h = ctypes.c_void_p()
        st = self.lib.sip_ctx_create(int(device), ctypes.byref(h))
        if st != _lib.SIP_OK:
            raise SipError(st, "sip_ctx_create failed")
        self.handle = h
        self.device = device

    def check(self, st):
        if st != _lib.SIP_OK:
            raise SipError(st, self.lib.sip_last_error(self.handle).decode())

    def close(self):
        if self.handle:
            self.lib.sip_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def rasterise_inclusions(self, nx, ny, shapes, eta_bg=1.0, rho_bg=1.0, lx=1.0, ly=1.0,
                             stream=None):
        """sip_rasterise_inclusions -> (eta, rho) as FP64 CUDA tensors.
        shapes: rows (kind, a, b, c, d, eta_i, rho_i)."""
        s = np.ascontiguousarray(np.asarray(shapes, dtype=np.float64).reshape(-1, 7))
        eta = torch.empty(nx * ny, dtype=torch.float64, device=f"cuda:{self.device}")
        rho = torch.empty_like(eta)
        self.check(self.lib.sip_rasterise_inclusions(
            self.handle, nx, ny, lx, ly, s.ctypes.data_as(ctypes.c_void_p), s.shape[0],
            eta_bg, rho_bg, _ptr(eta, torch.float64), _ptr(rho, torch.float64), _stream(stream)))
        return eta, rho


class Problem:
    """sip_problem: a discretised Stokes problem on the device."""

    def __init__(self, ctx, nx, ny, k, eta, bc=("navier",) * 4, lx=1.0, ly=1.0,
                 penalty_scale=1.0, n_hlevels=0, cheb_steps_p=2, cheb_steps_h=3,
                 eig_iters=10, cheb_lo=0.1, cheb_hi=1.1, seed=0, precision="fp64"):
        self.ctx = ctx
        lib = ctx.lib
        d = ProblemDesc()
        lib.sip_problem_desc_default(ctypes.byref(d))
        eta = np.ascontiguousarray(np.asarray(eta, dtype=np.float64).reshape(-1))
        self._eta = eta
        d.nx, d.ny, d.lx, d.ly, d.k = nx, ny, lx, ly, k
        for i, b in enumerate(bc):
            d.bc[i] = BC[b] if isinstance(b, str) else int(b)
        d.eta_host = eta.ctypes.data_as(_lib.c_double_p)
        d.penalty_scale = penalty_scale
        d.n_hlevels = n_hlevels
        d.cheb_steps_p, d.cheb_steps_h, d.eig_iters = cheb_steps_p, cheb_steps_h, eig_iters
        d.cheb_lo, d.cheb_hi = cheb_lo, cheb_hi
        d.seed = seed
        d.precision = PREC[precision] if isinstance(precision, str) else int(precision)
        h = ctypes.c_void_p()
        ctx.check(lib.sip_problem_create(ctx.handle, ctypes.byref(d), ctypes.byref(h)))
        self.handle = h
        self.nx, self.ny, self.k = nx, ny, k
        n_u, n_p, nbytes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        ctx.check(lib.sip_problem_sizes(h, ctypes.byref(n_u), ctypes.byref(n_p), ctypes.byref(nbytes)))
        self.n_u, self.n_p = n_u.value, n_p.value
        self.device = f"cuda:{ctx.device}"

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.sip_problem_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def device_bytes(self):
        n_u, n_p, nbytes = ctypes.c_int64(), ctypes.c_int64(), ctypes.c_int64()
        self.ctx.check(self.ctx.lib.sip_problem_sizes(self.handle, ctypes.byref(n_u),
                                                      ctypes.byref(n_p), ctypes.byref(nbytes)))
        return nbytes.value

    # -- operators ---------------------------------------------------------
    def apply_A(self, x, y, stream=None):
        self.ctx.check(self.ctx.lib.sip_apply_A(self.handle, _ptr(x, torch.float64),
                                                _ptr(y, torch.float64), _stream(stream)))

    def apply_A_f32(self, x, y, stream=None):
        self.ctx.check(self.ctx.lib.sip_apply_A_f32(self.handle, _ptr(x, torch.float32),
                                                    _ptr(y, torch.float32), _stream(stream)))

    def apply_B(self, xp, yu, stream=None):
        self.ctx.check(self.ctx.lib.sip_apply_B(self.handle, _ptr(xp, torch.float64),
                                                _ptr(yu, torch.float64), _stream(stream)))

    def apply_Bt(self, xu, yp, stream=None):
        self.ctx.check(self.ctx.lib.sip_apply_Bt(self.handle, _ptr(xu, torch.float64),
                                                 _ptr(yp, torch.float64), _stream(stream)))

    def rhs_body_force(self, rho, g, f, stream=None):
        self.ctx.check(self.ctx.lib.sip_rhs_body_force(self.handle, _ptr(rho, torch.float64),
                                                       float(g), _ptr(f, torch.float64),
                                                       _stream(stream)))
