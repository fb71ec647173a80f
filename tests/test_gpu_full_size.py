"""The many-disc workload at full size (512^2, k = 4, 64 discs of radius 0.02,
log10 eta ~ U[0, 6]), solved by the GPU in the FP64 and in the mixed form with
refinement by a double-double residual, checked against the oracle element by
element on sampled elements: the oracle rebuilds the rows of A, B and B^T of
each sampled element (corners, edges, tile seams, viscosity jumps) on their
own and evaluates the residual there, which must equal the GPU's residual of
the same result; the GPU residual over the whole mesh must meet the
tolerance (1e-8 in double-double, the FP64 evaluation within its rounding
floor at this contrast)."""
import numpy as np
import pytest
import torch

from oracle import sip
from paper_1607_03777_gb300 import api, synth

pytestmark = pytest.mark.gpu

N_MESH, K = 512, 4


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def sampled_elements(eta, n):
    """Corners, edge midpoints, warp-tile seams and the first viscosity jumps
    along x and along y."""
    E = eta.reshape(n, n)
    picks = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (n // 2, 0), (0, n // 3),
             (n - 1, n // 2), (n // 2, n - 1), (31, 3), (32, 4), (63, 7), (64, 8),
             (n // 2 + 1, n // 2 - 3)]
    jx = np.argwhere(E != np.roll(E, 1, axis=1))[:3]
    jy = np.argwhere(E != np.roll(E, 1, axis=0))[:3]
    picks += [(int(c), int(r)) for r, c in jx] + [(int(c), int(r)) for r, c in jy]
    return picks


def oracle_rows(ref, u, p, ex, ey):
    """(A u + B p) on the velocity dofs and (B^T u) on the pressure dofs of
    element (ex, ey), from element rows the oracle builds on their own, each
    with the sum of its terms' magnitudes (the scale of its FP64 rounding)."""
    num = ref.num
    nb, mp = num.nb, num.mp
    e = num.elem(ex, ey)
    au, au_abs = np.zeros(nb), np.zeros(nb)
    for f, blk in sip.element_rows_A(ref, ex, ey).items():
        au += blk @ u[f * nb:(f + 1) * nb]
        au_abs += np.abs(blk) @ np.abs(u[f * nb:(f + 1) * nb])
    bp, bp_abs = np.zeros(nb), np.zeros(nb)
    for f, blk in sip.element_rows_B(ref, ex, ey).items():
        bp += blk @ p[f * mp:(f + 1) * mp]
        bp_abs += np.abs(blk) @ np.abs(p[f * mp:(f + 1) * mp])
    btu, btu_abs = np.zeros(mp), np.zeros(mp)   # column e of B: rows of e and its neighbours
    for nbr in [(ex, ey)] + [sip.neighbour(ref, ex, ey, side) for side in sip.SIDES]:
        if nbr is None:
            continue
        f = num.elem(*nbr)
        blk = sip.element_rows_B(ref, *nbr).get(e)
        if blk is not None:
            btu += blk.T @ u[f * nb:(f + 1) * nb]
            btu_abs += np.abs(blk.T) @ np.abs(u[f * nb:(f + 1) * nb])
    return (au, au_abs), (bp, bp_abs), (btu, btu_abs)


@pytest.fixture(scope="module")
def field(ctx):
    wl = synth.many_discs(n=N_MESH, k=K, n_hlevels=synth.levels_to_17(N_MESH))
    eta_d, rho_d = ctx.rasterise_inclusions(N_MESH, N_MESH, wl.shapes)
    return wl, eta_d.cpu().numpy(), rho_d


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_many_discs_full_size_sampled(ctx, field, precision):
    wl, eta, rho_d = field
    n = N_MESH
    prob = api.Problem(ctx, n, n, K, eta, bc=wl.bc, n_hlevels=wl.n_hlevels, seed=1,
                       precision=precision)
    f = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    prob.rhs_body_force(rho_d, synth.GRAVITY, f)
    u_dd = torch.empty(2 * prob.n_u, dtype=torch.float64, device="cuda")
    p_dd = torch.empty(2 * prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve_dd(f, u_dd, p_dd, rtol=1e-8, max_outer=2000, max_inner=20, refine=4)
    assert rep["status"] == 0 and rep["rel_residual"] <= 1e-8, rep

    def rel_res_dd(xu, xp):
        ru, rp = torch.empty_like(xu), torch.empty_like(xp)
        prob.residual_dd(f, xu, xp, ru, rp)
        ru, rp = ru.view(-1, 2).sum(1), rp.view(-1, 2).sum(1)
        return float(torch.sqrt(torch.sum(ru * ru) + torch.sum(rp * rp)) / torch.linalg.norm(f))

    # the returned double-double iterate meets the tolerance, recomputed here
    rel_dd = rel_res_dd(u_dd, p_dd)
    assert rel_dd <= 1.001e-8, (precision, rel_dd)
    # rounded to FP64 it cannot: ||K|| eps_64 ||x|| is about 1e-7 ||b|| on this
    # field (contrast 1e6); the FP64 evaluation of the residual adds its own
    # rounding of the same size
    u = u_dd.view(-1, 2).sum(1)
    p = p_dd.view(-1, 2).sum(1)
    rel_rounded = rel_res_dd(torch.stack([u, torch.zeros_like(u)], 1).reshape(-1),
                             torch.stack([p, torch.zeros_like(p)], 1).reshape(-1))
    au, bp, btu = torch.empty_like(f), torch.empty_like(f), torch.empty_like(p)
    prob.apply_A(u, au)
    prob.apply_B(p, bp)
    prob.apply_Bt(u, btu)
    ru = f - au - bp
    rel64 = float(torch.sqrt(torch.sum(ru * ru) + torch.sum(btu * btu)) / torch.linalg.norm(f))
    print(f"{precision}: double-double iterate {rel_dd:.3e}, rounded to FP64 {rel_rounded:.3e}, "
          f"FP64 evaluation {rel64:.3e}")
    assert rel_rounded < 1e-6 and rel64 < 1e-6, (precision, rel_rounded, rel64)

    # sampled elements: the oracle's rows against the GPU's operators, to a
    # small multiple of FP64 rounding on the element's largest sum of term
    # magnitudes (structurally zero entries carry quadrature noise)
    ref = sip.Problem(n, n, K, eta, bc=wl.bc)
    uh, ph, fh = host(u), host(p), host(f)
    auh, bph, btuh, ruh = host(au), host(bp), host(btu), host(ru)
    nb, mp = ref.num.nb, ref.num.mp
    tol = 1e-12
    for ex, ey in sampled_elements(eta, n):
        e = ref.num.elem(ex, ey)
        (a_o, a_s), (b_o, b_s), (t_o, t_s) = oracle_rows(ref, uh, ph, ex, ey)
        su, sp = slice(e * nb, (e + 1) * nb), slice(e * mp, (e + 1) * mp)
        assert np.abs(auh[su] - a_o).max() <= tol * a_s.max(), (precision, ex, ey)
        assert np.abs(bph[su] - b_o).max() <= tol * b_s.max(), (precision, ex, ey)
        assert np.abs(btuh[sp] - t_o).max() <= tol * t_s.max(), (precision, ex, ey)
        # the residual of this element from the oracle's rows is the GPU's
        r_o = fh[su] - a_o - b_o
        assert np.abs(ruh[su] - r_o).max() <= tol * (a_s + b_s + np.abs(fh[su])).max(), \
            (precision, ex, ey)
