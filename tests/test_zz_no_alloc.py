"""The allocation-free rasteriser (sip_rasterise_inclusions_noalloc).

Some callers cannot call cudaMalloc: code embedded in a framework that owns
all device memory through its own pool and budget, or a latency-bound loop in
which an allocation or free would synchronise the device.  For them the
library stages the inclusion records in a fixed device array compiled into
the library instead of a fresh allocation.  This file checks, through the C
ABI, that two calls in a row give exactly what the allocating entry point
gives, and that a list longer than the array is refused.  It is collected
last, and passes both alone and after the other tests.
"""
import ctypes

import numpy as np
import pytest
import torch

from paper_1607_03777_gb300 import _lib, synth

pytestmark = pytest.mark.gpu

MAX_SHAPES = 4096   # SIP_NOALLOC_MAX_SHAPES in include/sipstokes.h


def _noalloc(ctx, nx, ny, shapes, eta_bg=1.0, rho_bg=1.0):
    lib = _lib.load()
    s = np.ascontiguousarray(np.asarray(shapes, dtype=np.float64).reshape(-1, 7))
    eta = torch.full((nx * ny,), -1.0, dtype=torch.float64, device="cuda")
    rho = torch.full_like(eta, -1.0)
    stream = torch.cuda.current_stream()
    st = lib.sip_rasterise_inclusions_noalloc(
        ctx.handle, nx, ny, 1.0, 1.0, s.ctypes.data_as(ctypes.c_void_p), s.shape[0], eta_bg,
        rho_bg, ctypes.c_void_p(eta.data_ptr()), ctypes.c_void_p(rho.data_ptr()),
        ctypes.c_void_p(stream.cuda_stream))
    torch.cuda.synchronize()
    return st, eta, rho


def test_noalloc_matches_allocating_entry_point_twice(ctx):
    cases = [
        (96, 80, np.concatenate([synth.random_discs(64, 0.02, (0.0, 6.0), seed=3),
                                 np.stack([synth.box(0.25, 0.75, 0.25, 0.75, 1e4, 1.2)])])),
        (33, 47, synth.random_discs(7, 0.09, (1.0, 3.0), seed=11)),   # fewer records than before
        (5, 3, np.zeros((0, 7))),     # no record at all: the stale ones must not be read
    ]
    for nx, ny, shapes in cases:
        bg = (2.0, 0.5) if len(shapes) == 0 else (1.0, 1.0)
        st, eta, rho = _noalloc(ctx, nx, ny, shapes, *bg)
        assert st == _lib.SIP_OK, ctx.lib.sip_last_error(ctx.handle).decode()
        eta_ref, rho_ref = ctx.rasterise_inclusions(nx, ny, shapes, eta_bg=bg[0], rho_bg=bg[1])
        torch.cuda.synchronize()
        assert torch.equal(eta, eta_ref)
        assert torch.equal(rho, rho_ref)


def test_noalloc_rejects_too_many_records(ctx):
    shapes = np.tile(synth.disc(0.5, 0.5, 0.1, 2.0, 1.0), (MAX_SHAPES + 1, 1))
    st, eta, _ = _noalloc(ctx, 8, 8, shapes)
    assert st == 1   # SIP_ERR_INVALID_ARG
    assert "at most" in ctx.lib.sip_last_error(ctx.handle).decode()
    assert (eta == -1.0).all()       # nothing was launched
    st, _, _ = _noalloc(ctx, 8, 8, shapes[:MAX_SHAPES])
    assert st == _lib.SIP_OK
