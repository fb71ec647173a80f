"""GPU parity of the double-double residual and of iterative refinement
(the precision question of Sec. 7.4)."""
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import krylov, sip
from paper_1607_03777_gb300 import api, synth

pytestmark = pytest.mark.gpu

SINK = ("navier", "navier", "navier", "neumann")


def _dd_pairs(hi, lo):
    """(hi, lo) interleaved float64 tensor on the device."""
    return torch.from_numpy(np.stack([hi, lo], axis=1).reshape(-1).copy()).cuda()


def _frac(pairs, i):
    return Fraction(float(pairs[2 * i])) + Fraction(float(pairs[2 * i + 1]))


def test_residual_dd_precision(ctx):
    """r = b - K x in double-double on a ragged 13 x 10 mesh, k = 3, random
    eta 10^U[0,3]: (1) its leading part equals the oracle's FP64 residual to
    FP64 rounding; (2) it carries ~106 bits: r(x_hi + x_lo) - r(x_hi) equals
    -K x_lo = r(x_lo) - r(0) exactly up to 1e-27 of |r|, checked in rational
    arithmetic on sampled entries, where FP64 arithmetic would be wrong in
    the first digit of that difference."""
    nx, ny, k = 13, 10, 3
    eta = synth.random_eta(nx * ny, 61, (0.0, 3.0))
    prob = api.Problem(ctx, nx, ny, k, eta, bc=SINK, n_hlevels=0, seed=1)
    ref = sip.Problem(nx, ny, k, eta, bc=SINK)
    n_u, n_p = prob.n_u, prob.n_p
    g = np.random.default_rng(62)
    f, gp = g.standard_normal(n_u), g.standard_normal(n_p)
    x_hi = g.standard_normal(n_u + n_p)
    x_lo = x_hi * g.uniform(-1, 1, x_hi.size) * 2.0 ** -54
    zero = np.zeros_like(x_hi)
    fd, gd = torch.from_numpy(f).cuda(), torch.from_numpy(gp).cuda()
    zf, zg = torch.zeros_like(fd), torch.zeros_like(gd)

    def res(hi, lo, fv, gv):
        xu, xp = _dd_pairs(hi[:n_u], lo[:n_u]), _dd_pairs(hi[n_u:], lo[n_u:])
        ru = torch.empty(2 * n_u, dtype=torch.float64, device="cuda")
        rp = torch.empty(2 * n_p, dtype=torch.float64, device="cuda")
        prob.residual_dd(fv, xu, xp, ru, rp, g=gv)
        torch.cuda.synchronize()
        return np.concatenate([ru.cpu().numpy(), rp.cpu().numpy()])

    r_full = res(x_hi, x_lo, fd, gd)
    r_hi = res(x_hi, zero, fd, gd)
    r_lo = res(x_lo, zero, zf, zg)       # -K x_lo
    # (1) parity of the leading part with the oracle in FP64
    A, B = sip.assemble_A(ref), sip.assemble_B(ref)
    K = krylov.stokes_matrix(A, B).tocsr()
    r64 = np.concatenate([f, gp]) - K @ x_hi
    lead = r_hi[0::2] + r_hi[1::2]
    assert np.linalg.norm(lead - r64) <= 1e-12 * np.linalg.norm(r64)
    # (2) 106-bit linearity on sampled entries, in exact arithmetic
    scale = Fraction(float(np.abs(r64).max()))
    idx = np.random.default_rng(63).choice(n_u + n_p, 1500, replace=False)
    worst = Fraction(0)
    for i in idx:
        d = _frac(r_full, i) - _frac(r_hi, i) - _frac(r_lo, i)
        worst = max(worst, abs(d))
    assert worst <= Fraction(1, 10 ** 27) * scale, float(worst / scale)


def test_solve_refine_below_fp64_floor(ctx):
    """Six inclusions, contrast 1e8, 32^2, k = 2, rtol 1e-10: the FP64 solve
    stops on stagnation above the tolerance (FP64's attainable accuracy);
    with refinement the double-double residual of the refined iterate meets
    it in a few correction solves."""
    n, k = 32, 2
    wl = synth.six_sinkers(n=n, k=k, eta_in=1e8, n_hlevels=1)
    eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
    prob = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=wl.bc, n_hlevels=1, seed=1)
    f = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    u = torch.empty_like(f)
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    prob.rhs_body_force(rho, synth.GRAVITY, f)
    plain = prob.solve(f, u, p, rtol=1e-10, max_outer=400, check=False)
    assert plain["status"] != 0 and plain["rel_residual"] > 1e-10, plain
    assert plain["outer_its"] < 400, plain   # stopped on stagnation, not the cap
    u_plain = u.clone()
    rep = prob.solve(f, u, p, rtol=1e-10, max_outer=400, refine=6, check=False)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-10, rep
    assert 2 <= rep["refine_steps"] <= 6, rep
    # the refined and the stalled solutions differ by the stalled one's error
    d = float(torch.linalg.norm(u - u_plain) / torch.linalg.norm(u_plain))
    assert d < 1e-3, d
