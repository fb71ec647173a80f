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
from ._lib import SipError, ProblemDesc, SolveOpts, SolveReport, BC, PREC, COARSE


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
                 eig_iters=10, cheb_lo=0.1, cheb_hi=1.1, seed=0, precision="fp64",
                 coarse="q1", mixed_fp64_ratio=1e3):
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
        d.coarse = COARSE[coarse] if isinstance(coarse, str) else int(coarse)
        d.mixed_fp64_ratio = float(mixed_fp64_ratio)
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

    def schedule(self):
        """sip_problem_schedule: {"apply": [fp64, fp32], "fused": [fp64, fp32]}
        (apply: 1 component split, 2 one thread per element, 3 tile, 4 / 5
        staged tile with 2 / 4 rows)."""
        apply = (ctypes.c_int * 2)()
        fused = (ctypes.c_int * 2)()
        self.ctx.check(self.ctx.lib.sip_problem_schedule(self.handle, apply, fused))
        return {"apply": list(apply), "fused": list(fused)}

    def set_schedule(self, apply=None, fused=None):
        """sip_problem_set_schedule: pin the apply kernel ([fp64, fp32] codes
        of ``schedule``, 0 = autotuned) and the fused smoother step ([fp64,
        fp32], -1 = autotuned); None leaves a pair unchanged."""
        a = (ctypes.c_int * 2)(*apply) if apply is not None else None
        f = (ctypes.c_int * 2)(*fused) if fused is not None else None
        self.ctx.check(self.ctx.lib.sip_problem_set_schedule(self.handle, a, f))

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

    def residual_dd(self, f, x_u, x_p, r_u, r_p, g=None, stream=None):
        """sip_residual_dd: r = b - K x in double-double; x_u, x_p, r_u, r_p
        are float64 tensors of 2 n_u / 2 n_p entries, (hi, lo) pairs."""
        for t, m in ((x_u, self.n_u), (x_p, self.n_p), (r_u, self.n_u), (r_p, self.n_p)):
            if t.numel() != 2 * m:
                raise ValueError("double-double vectors hold 2 doubles per entry")
        self.ctx.check(self.ctx.lib.sip_residual_dd(
            self.handle, _ptr(f, torch.float64),
            _ptr(g, torch.float64) if g is not None else None, _ptr(x_u, torch.float64),
            _ptr(x_p, torch.float64), _ptr(r_u, torch.float64), _ptr(r_p, torch.float64),
            _stream(stream)))

    def rhs_body_force(self, rho, g, f, stream=None):
        self.ctx.check(self.ctx.lib.sip_rhs_body_force(self.handle, _ptr(rho, torch.float64),
                                                       float(g), _ptr(f, torch.float64),
                                                       _stream(stream)))

    def update_eta(self, eta, stream=None):
        """sip_problem_update_eta with a CUDA tensor or a host array."""
        if isinstance(eta, torch.Tensor):
            ptr = _ptr(eta, torch.float64)
        else:
            self._eta = np.ascontiguousarray(np.asarray(eta, dtype=np.float64).reshape(-1))
            ptr = self._eta.ctypes.data_as(ctypes.c_void_p)
        self.ctx.check(self.ctx.lib.sip_problem_update_eta(self.handle, ptr, _stream(stream)))

    # -- hp-multigrid pieces -------------------------------------------------
    def setup(self, stream=None):
        self.ctx.check(self.ctx.lib.sip_problem_setup(self.handle, _stream(stream)))

    def lambda_max(self, level=-1):
        out = ctypes.c_double()
        self.ctx.check(self.ctx.lib.sip_lambda_max(self.handle, int(level), ctypes.byref(out)))
        return out.value

    def _call4(self, name, a, b, dta=torch.float64, dtb=torch.float64, stream=None):
        fn = getattr(self.ctx.lib, name)
        self.ctx.check(fn(self.handle, _ptr(a, dta), _ptr(b, dtb), _stream(stream)))

    def block_jacobi(self, r, z, stream=None):
        self._call4("sip_block_jacobi", r, z, stream=stream)

    def p_restrict(self, r, r1, stream=None):
        self._call4("sip_p_restrict", r, r1, stream=stream)

    def p_prolong_add(self, e1, y, stream=None):
        self._call4("sip_p_prolong_add", e1, y, stream=stream)

    def apply_A1(self, x1, y1, stream=None):
        self._call4("sip_apply_A1", x1, y1, stream=stream)

    def cd_prolong(self, v, u1, stream=None):
        self._call4("sip_cd_prolong", v, u1, stream=stream)

    def dc_restrict(self, u1, v, stream=None):
        self._call4("sip_dc_restrict", u1, v, stream=stream)

    def hlevel_dims(self, level=0):
        nl, nvx, nvy = ctypes.c_int(), ctypes.c_int(), ctypes.c_int()
        self.ctx.check(self.ctx.lib.sip_hlevel_dims(self.handle, int(level), ctypes.byref(nl),
                                                    ctypes.byref(nvx), ctypes.byref(nvy)))
        return nl.value, nvx.value, nvy.value

    def hlevel_stencil(self, level, S, stream=None):
        self.ctx.check(self.ctx.lib.sip_hlevel_stencil(self.handle, int(level),
                                                       _ptr(S, torch.float64), _stream(stream)))

    def hlevel_apply(self, level, x, y, stream=None):
        self.ctx.check(self.ctx.lib.sip_hlevel_apply(self.handle, int(level), _ptr(x, torch.float64),
                                                     _ptr(y, torch.float64), _stream(stream)))

    def coarse_solve(self, b, x, stream=None):
        self._call4("sip_coarse_solve", b, x, stream=stream)

    def vcycle(self, r, z, stream=None):
        self._call4("sip_vcycle", r, z, stream=stream)

    def vcycle_f32(self, r, z, stream=None):
        self._call4("sip_vcycle_f32", r, z, torch.float32, torch.float32, stream=stream)

    def inner_solve(self, t, y, rtol=1e-3, max_it=200, stream=None):
        its = ctypes.c_int()
        self.ctx.check(self.ctx.lib.sip_inner_solve(self.handle, _ptr(t, torch.float64),
                                                    _ptr(y, torch.float64), float(rtol), int(max_it),
                                                    ctypes.byref(its), _stream(stream)))
        return its.value

    # -- Stokes solve --------------------------------------------------------
    def solve(self, f, u, p, g=None, rtol=1e-8, max_outer=500, restart=100, inner_rtol=1e-3,
              max_inner=200, inner_loop="device", inner_krylov="auto",
              inner_norm="true", inner_restart=30, outer_krylov="fgmres", refine=0,
              time_limit_ms=0.0, stream=None, check=True):
        """sip_solve; returns the report as a dict (raises on failure when
        ``check``).  ``inner_loop`` = "device" (one graph launch per inner
        solve) or "host" (host-driven loop); ``inner_krylov`` = "auto",
        "pcg", "fcg" or "gcr" (restarted after ``inner_restart`` directions,
        device loop only); ``inner_norm`` = "true" (the residual, the
        default; GCR always tests it) or "preconditioned" (the V-cycle
        applied to the residual; device loop only); ``outer_krylov`` =
        "fgmres" (default) or "gcr"; ``refine`` = the most correction solves
        of iterative refinement with a double-double residual (0: off);
        ``time_limit_ms`` > 0 stops the solve between outer iterations once
        that much wall time has passed (status SIP_ERR_TIMEOUT)."""
        o = _opts(self.ctx.lib, rtol, max_outer, restart, inner_rtol, max_inner, inner_loop,
                  inner_krylov, inner_norm, inner_restart, outer_krylov, refine, time_limit_ms)
        rep = SolveReport()
        st = self.ctx.lib.sip_solve(self.handle, _ptr(f, torch.float64),
                                    _ptr(g, torch.float64) if g is not None else None,
                                    _ptr(u, torch.float64), _ptr(p, torch.float64),
                                    ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        out = {name: getattr(rep, name) for name, _ in SolveReport._fields_}
        if check:
            self.ctx.check(st)
        out["status"] = st
        return out

    def solve_dd(self, f, u_dd, p_dd, g=None, rtol=1e-8, max_outer=500, restart=100,
                 inner_rtol=1e-3, max_inner=200, inner_loop="device", inner_krylov="auto",
                 inner_norm="true", inner_restart=30, outer_krylov="fgmres", refine=4,
                 time_limit_ms=0.0, stream=None, check=True):
        """sip_solve_dd: the refined solve (``refine`` > 0) returning its
        double-double iterate in ``u_dd``, ``p_dd`` (float64 tensors of
        2 n_u / 2 n_p entries, (hi, lo) pairs); options and report as
        ``solve``."""
        for t, m in ((u_dd, self.n_u), (p_dd, self.n_p)):
            if t.numel() != 2 * m:
                raise ValueError("double-double vectors hold 2 doubles per entry")
        o = _opts(self.ctx.lib, rtol, max_outer, restart, inner_rtol, max_inner, inner_loop,
                  inner_krylov, inner_norm, inner_restart, outer_krylov, refine, time_limit_ms)
        rep = SolveReport()
        st = self.ctx.lib.sip_solve_dd(self.handle, _ptr(f, torch.float64),
                                       _ptr(g, torch.float64) if g is not None else None,
                                       _ptr(u_dd, torch.float64), _ptr(p_dd, torch.float64),
                                       ctypes.byref(o), ctypes.byref(rep), _stream(stream))
        out = {name: getattr(rep, name) for name, _ in SolveReport._fields_}
        if check:
            self.ctx.check(st)
        out["status"] = st
        return out


# ---------------------------------------------------------------- batches, serving
def make_desc(ctx, nx, ny, k, eta, bc=("navier",) * 4, lx=1.0, ly=1.0, penalty_scale=1.0,
              n_hlevels=0, cheb_steps_p=2, cheb_steps_h=3, eig_iters=10, cheb_lo=0.1,
              cheb_hi=1.1, seed=0, precision="fp64", coarse="q1", mixed_fp64_ratio=1e3):
    """A filled sip_problem_desc and the host eta array it points to (keep
    both alive while the C side may read them)."""
    d = ProblemDesc()
    ctx.lib.sip_problem_desc_default(ctypes.byref(d))
    eta = np.ascontiguousarray(np.asarray(eta, dtype=np.float64).reshape(-1))
    d.nx, d.ny, d.lx, d.ly, d.k = nx, ny, lx, ly, k
    for i, b in enumerate(bc):
        d.bc[i] = BC[b] if isinstance(b, str) else int(b)
    d.eta_host = eta.ctypes.data_as(_lib.c_double_p)
    d.penalty_scale, d.n_hlevels = penalty_scale, n_hlevels
    d.cheb_steps_p, d.cheb_steps_h, d.eig_iters = cheb_steps_p, cheb_steps_h, eig_iters
    d.cheb_lo, d.cheb_hi, d.seed = cheb_lo, cheb_hi, seed
    d.precision = PREC[precision] if isinstance(precision, str) else int(precision)
    d.coarse = COARSE[coarse] if isinstance(coarse, str) else int(coarse)
    d.mixed_fp64_ratio = float(mixed_fp64_ratio)
    return d, eta


INNER_LOOP = {"device": 0, "host": 1}
INNER_KRYLOV = {"auto": 0, "pcg": 1, "fcg": 2, "gcr": 3}
INNER_NORM = {"true": 0, "preconditioned": 1}
OUTER_KRYLOV = {"fgmres": 0, "gcr": 1}


def _opts(lib, rtol=1e-8, max_outer=500, restart=100, inner_rtol=1e-3, max_inner=200,
          inner_loop="device", inner_krylov="auto", inner_norm="true",
          inner_restart=30, outer_krylov="fgmres", refine=0, time_limit_ms=0.0):
    o = SolveOpts()
    lib.sip_solve_opts_default(ctypes.byref(o))
    o.rtol, o.max_outer, o.restart = rtol, max_outer, restart
    o.inner_rtol, o.max_inner = inner_rtol, max_inner
    o.inner_loop = INNER_LOOP[inner_loop] if isinstance(inner_loop, str) else int(inner_loop)
    o.inner_krylov = (INNER_KRYLOV[inner_krylov] if isinstance(inner_krylov, str)
                      else int(inner_krylov))
    o.inner_norm = INNER_NORM[inner_norm] if isinstance(inner_norm, str) else int(inner_norm)
    o.inner_restart = int(inner_restart)
    o.outer_krylov = (OUTER_KRYLOV[outer_krylov] if isinstance(outer_krylov, str)
                      else int(outer_krylov))
    o.refine = int(refine)
    o.time_limit_ms = float(time_limit_ms)
    return o


def _report(rep):
    return {name: getattr(rep, name) for name, _ in SolveReport._fields_}


def footprint(ctx, restart=100, **desc_kw):
    d, _keep = make_desc(ctx, **desc_kw)
    return int(ctx.lib.sip_problem_footprint(ctypes.byref(d), int(restart)))


def solve_batch(ctx, problems, fs, us, ps, n_streams=8, stream=None, grouped=False, **opt_kw):
    """sip_solve_batch (or, with ``grouped``, sip_solve_batch_grouped with
    groups of ``n_streams`` problems) over lists of Problems and CUDA
    tensors; returns (status, [report dicts])."""
    n = len(problems)
    arr = lambda vals: (ctypes.c_void_p * n)(*vals)
    hp = arr([p.handle.value for p in problems])
    hf = arr([_ptr(f, torch.float64).value for f in fs])
    hu = arr([_ptr(u, torch.float64).value for u in us])
    hpp = arr([_ptr(p, torch.float64).value for p in ps])
    reps = (SolveReport * n)()
    o = _opts(ctx.lib, **opt_kw)
    torch.cuda.current_stream().synchronize()
    fn = ctx.lib.sip_solve_batch_grouped if grouped else ctx.lib.sip_solve_batch
    st = fn(ctx.handle, n, hp, hf, hu, hpp, ctypes.byref(o), reps, int(n_streams))
    return st, [_report(r) for r in reps]


class Server:
    """sip_server: continuous batching of Stokes solve requests."""

    def __init__(self, ctx, budget_bytes, max_slots=8):
        self.ctx = ctx
        h = ctypes.c_void_p()
        ctx.check(ctx.lib.sip_server_create(ctx.handle, int(budget_bytes), int(max_slots),
                                            ctypes.byref(h)))
        self.handle = h
        self._keep = {}

    def submit(self, request_id, nx, ny, k, eta, rho, g=10.0, opts=None, **desc_kw):
        """Queue a request; returns (status, u_host, p_host) with the host
        output arrays that the server fills."""
        d, eta_keep = make_desc(self.ctx, nx, ny, k, eta, **desc_kw)
        rho = np.ascontiguousarray(np.asarray(rho, dtype=np.float64).reshape(-1))
        n = k + 1
        u = np.zeros(nx * ny * 2 * n * n)
        p = np.zeros(nx * ny * k * k)
        o = _opts(self.ctx.lib, **(opts or {}))
        st = self.ctx.lib.sip_server_submit(self.handle, ctypes.byref(d),
                                            rho.ctypes.data_as(ctypes.c_void_p), float(g),
                                            u.ctypes.data_as(ctypes.c_void_p),
                                            p.ctypes.data_as(ctypes.c_void_p), ctypes.byref(o),
                                            ctypes.c_uint64(request_id))
        self._keep[request_id] = (u, p)
        return st, u, p

    def poll(self, cap=256):
        ids = (ctypes.c_uint64 * cap)()
        reps = (SolveReport * cap)()
        n = ctypes.c_int()
        self.ctx.check(self.ctx.lib.sip_server_poll(self.handle, ids, reps, cap, ctypes.byref(n)))
        out = []
        for i in range(n.value):
            out.append((int(ids[i]), _report(reps[i])))
            self._keep.pop(int(ids[i]), None)
        return out

    def cancel(self, request_id):
        """sip_server_cancel; returns the status (SIP_OK, or
        SIP_ERR_INVALID_ARG for an id that is neither queued nor running)."""
        return self.ctx.lib.sip_server_cancel(self.handle, ctypes.c_uint64(request_id))

    def drain(self):
        self.ctx.check(self.ctx.lib.sip_server_drain(self.handle))

    def stats(self):
        q, r, b = ctypes.c_int(), ctypes.c_int(), ctypes.c_int64()
        self.ctx.check(self.ctx.lib.sip_server_stats(self.handle, ctypes.byref(q), ctypes.byref(r),
                                                     ctypes.byref(b)))
        return {"queued": q.value, "running": r.value, "bytes_in_use": b.value}

    def close(self):
        if getattr(self, "handle", None):
            self.ctx.lib.sip_server_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
