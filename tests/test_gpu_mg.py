"""GPU parity of the hp-multigrid pieces, the inner PCG and the Stokes solve
against the FP64 oracle, through the C ABI."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla
import torch

from oracle import exact, krylov, materials, multigrid, sip
from paper_1607_03777_gb300 import api, synth

pytestmark = pytest.mark.gpu

SINK = synth.SINKER_BC
BCS = [("navier",) * 4, SINK, ("dirichlet",) * 4, ("neumann", "dirichlet", "navier", "neumann")]


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def pair(ctx, nx, ny, k, bc, eta, nh=0, seed=3, precision="fp64", coarse="q1"):
    prob = api.Problem(ctx, nx, ny, k, eta, bc=bc, n_hlevels=nh, seed=seed, precision=precision,
                       coarse=coarse)
    ref = sip.Problem(nx, ny, k, eta, bc=bc)
    return prob, ref


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
def test_block_jacobi(ctx, k):
    for i, bc in enumerate(BCS):
        nx, ny = 5, 4
        eta = synth.random_eta(nx * ny, 40 + i, (0.0, 3.0))
        eta[3] = eta.max() * 2       # a class element next to unique ones
        prob, ref = pair(ctx, nx, ny, k, bc, eta)
        A = sip.assemble_A(ref)
        inv = multigrid.invert_blocks(multigrid.block_jacobi_blocks(A, ref.num.nb))
        r = synth.random_vector(prob.n_u, 50 + i)
        z = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        prob.block_jacobi(dev(r), z)
        assert rel(host(z), multigrid.block_apply(inv, r)) < 1e-9, bc


def test_block_jacobi_uniform_eta_uses_classes(ctx):
    """All elements share one viscosity: every block is a scaled reference
    block (class path) and the result still matches the oracle."""
    for bc in BCS[:2]:
        prob, ref = pair(ctx, 6, 6, 3, bc, np.full(36, 7.5))
        A = sip.assemble_A(ref)
        inv = multigrid.invert_blocks(multigrid.block_jacobi_blocks(A, ref.num.nb))
        r = synth.random_vector(prob.n_u, 1)
        z = torch.empty_like(dev(r))
        prob.block_jacobi(dev(r), z)
        assert rel(host(z), multigrid.block_apply(inv, r)) < 1e-10


@pytest.mark.parametrize("k", [1, 2, 4])
def test_lambda_max_p(ctx, k):
    nx = ny = 6
    eta = synth.random_eta(nx * ny, 7, (0.0, 2.0))
    prob, ref = pair(ctx, nx, ny, k, SINK, eta, seed=11)
    A = sip.assemble_A(ref)
    inv = multigrid.invert_blocks(multigrid.block_jacobi_blocks(A, ref.num.nb))
    lam_ref = multigrid.estimate_lambda_max(lambda v: A @ v, lambda v: multigrid.block_apply(inv, v),
                                            A.shape[0], seed=11)
    assert abs(prob.lambda_max(-1) - lam_ref) < 1e-9 * lam_ref


def test_p_transfers_exact(ctx):
    prob, _ = pair(ctx, 4, 3, 3, SINK, np.ones(12))
    r = synth.random_vector(prob.n_u, 3)
    r1 = torch.empty(12 * 8, dtype=torch.float64, device="cuda")
    prob.p_restrict(dev(r), r1)
    P = multigrid.p_prolongation(3, 12, 1)
    assert np.array_equal(host(r1), P.T @ r)
    y = dev(r)
    e1 = synth.random_vector(96, 4)
    prob.p_prolong_add(dev(e1), y)
    assert np.array_equal(host(y), r + P @ e1)


@pytest.mark.parametrize("k", [1, 3, 6])
def test_apply_A1_galerkin(ctx, k):
    for bc in BCS:
        nx, ny = 5, 3
        eta = synth.random_eta(nx * ny, k, (0.0, 3.0))
        prob, ref = pair(ctx, nx, ny, k, bc, eta)
        A = sip.assemble_A(ref)
        P = multigrid.p_prolongation(k, nx * ny, 1)
        A1 = P.T @ A @ P
        x = synth.random_vector(nx * ny * 8, 9)
        y = torch.empty(nx * ny * 8, dtype=torch.float64, device="cuda")
        prob.apply_A1(dev(x), y)
        assert rel(host(y), A1 @ x) < 1e-10, bc


def test_pcd_rdc(ctx):
    nx, ny = 6, 5
    prob, _ = pair(ctx, nx, ny, 2, SINK, np.ones(nx * ny))
    Pcd = multigrid.continuous_to_dg(nx, ny)
    v = synth.random_vector(2 * (nx + 1) * (ny + 1), 1)
    u1 = torch.empty(nx * ny * 8, dtype=torch.float64, device="cuda")
    prob.cd_prolong(dev(v), u1)
    assert rel(host(u1), Pcd @ v) < 1e-14
    w = synth.random_vector(nx * ny * 8, 2)
    vv = torch.empty(2 * (nx + 1) * (ny + 1), dtype=torch.float64, device="cuda")
    prob.dc_restrict(dev(w), vv)
    assert rel(host(vv), Pcd.T @ w) < 1e-14


@pytest.mark.parametrize("bc", [SINK, ("navier",) * 4, ("dirichlet",) * 4])
def test_hlevel_stencils_and_coarse(ctx, bc):
    nx = ny = 16
    k = 2
    eta, _ = materials.rasterise_inclusions(nx, ny, synth.single_box_inclusion(nx, k, 1e3).shapes)
    prob, ref = pair(ctx, nx, ny, k, bc, eta, nh=2, seed=5)
    A = sip.assemble_A(ref)
    mg = multigrid.HPMultigrid(ref, A, 2, seed=5)
    nl, _, _ = prob.hlevel_dims(0)
    assert nl == 3
    mats = [lv.A for lv in mg.h.levels] + [mg.h.coarse_A]
    for l in range(3):
        _, nvx, nvy = prob.hlevel_dims(l)
        x = synth.random_vector(2 * nvx * nvy, 20 + l)
        y = torch.empty_like(dev(x))
        prob.hlevel_apply(l, dev(x), y)
        assert rel(host(y), mats[l] @ x) < 1e-10, l
        if l < 2:
            assert abs(prob.lambda_max(l) - mg.h.levels[l].lmax) < 1e-9 * mg.h.levels[l].lmax
    # coarsest direct solve
    _, nvx, nvy = prob.hlevel_dims(2)
    b = synth.random_vector(2 * nvx * nvy, 5)
    x = torch.empty_like(dev(b))
    prob.coarse_solve(dev(b), x)
    assert rel(host(x), np.linalg.solve(mg.h.coarse_A, b)) < 1e-9


@pytest.mark.parametrize("nh,k,bc", [(0, 2, ("dirichlet",) * 4), (2, 3, SINK), (1, 2, ("navier",) * 4)])
def test_vcycle_fp64(ctx, nh, k, bc):
    nx = ny = 16
    eta, _ = materials.rasterise_inclusions(nx, ny, synth.single_box_inclusion(nx, k, 1e3).shapes)
    prob, ref = pair(ctx, nx, ny, k, bc, eta, nh=nh, seed=9)
    A = sip.assemble_A(ref)
    mg = multigrid.HPMultigrid(ref, A, nh, seed=9)
    assert abs(prob.lambda_max(-1) - mg.lmax) < 1e-9 * mg.lmax
    r = synth.random_vector(prob.n_u, 77)
    z = torch.empty_like(dev(r))
    prob.vcycle(dev(r), z)
    assert rel(host(z), mg(r)) < 1e-9
    prob.vcycle(dev(r), z)      # repeatable (graph replay)
    assert rel(host(z), mg(r)) < 1e-9


def test_vcycle_fp32(ctx):
    nx = ny = 16
    k = 3
    eta, _ = materials.rasterise_inclusions(nx, ny, synth.single_box_inclusion(nx, k, 1e3).shapes)
    prob, ref = pair(ctx, nx, ny, k, SINK, eta, nh=2, seed=9, precision="mixed")
    A = sip.assemble_A(ref)
    mg = multigrid.HPMultigrid(ref, A, 2, seed=9)
    r = synth.random_vector(prob.n_u, 78).astype(np.float32)
    z = torch.empty(prob.n_u, dtype=torch.float32, device="cuda")
    prob.vcycle_f32(dev(r, torch.float32), z)
    assert rel(host(z), mg(r.astype(np.float64))) < 2e-4


def test_inner_pcg(ctx):
    nx = ny = 16
    k = 2
    eta, rho = materials.rasterise_inclusions(nx, ny, synth.single_box_inclusion(nx, k, 1e2).shapes)
    prob, ref = pair(ctx, nx, ny, k, SINK, eta, nh=1, seed=2)
    A = sip.assemble_A(ref)
    mg = multigrid.HPMultigrid(ref, A, 1, seed=2)
    t = sip.rhs_body_force(ref, rho)
    y_ref, its_ref = krylov.pcg(lambda v: A @ v, mg, t, 1e-6, 200)
    y = torch.empty_like(dev(t))
    its = prob.inner_solve(dev(t), y, rtol=1e-6, max_it=200)
    assert abs(its - its_ref) <= 1
    assert np.linalg.norm(A @ host(y) - t) < 1e-6 * np.linalg.norm(t)
    assert rel(host(y), y_ref) < 1e-5


def _true_residual(ref, u, p, f):
    A, B = sip.assemble_A(ref), sip.assemble_B(ref)
    K = krylov.stokes_matrix(A, B)
    b = np.concatenate([f, np.zeros(B.shape[1])])
    x = np.concatenate([u, p])
    return np.linalg.norm(b - K @ x) / np.linalg.norm(b), A, B


def test_solve_dirichlet_mms_two_level(ctx):
    """8x8, k = 2, Dirichlet manufactured solution, A_p(Q^2_1) two-level
    preconditioner, rtol 1e-10: GPU solution = sparse-direct oracle solution."""
    sol = exact.SmoothDirichlet()
    nx = ny = 8
    prob, ref = pair(ctx, nx, ny, 2, ("dirichlet",) * 4, np.ones(64), nh=0, seed=7)
    f = sip.rhs_force(ref, sol.f)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-10)
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.5e-10, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-8
    assert rel(host(p), p_ref) < 1e-7    # p is less well conditioned than u
    assert abs(host(p)[::4].mean()) < 1e-12      # zero-mean pressure


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_box_inclusion(ctx, precision):
    """Single box inclusion 1e4 (Neumann top, Navier elsewhere), Q^2_1 + 1
    h-coarsening, rtol 1e-8: true FP64 residual (oracle matrices) <= 1e-8 and
    the solution matches the sparse-direct oracle."""
    nx = ny = 16
    k = 3
    wl = synth.single_box_inclusion(nx, k, 1e4, n_hlevels=1)
    eta, rho = materials.rasterise_inclusions(nx, ny, wl.shapes)
    prob, ref = pair(ctx, nx, ny, k, wl.bc, eta, nh=1, seed=1, precision=precision)
    f = sip.rhs_body_force(ref, rho)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-8, inner_rtol=1e-3, max_outer=1000)
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.05e-8, rep
    assert abs(rep["rel_residual"] - res) < 1e-9
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-5


@pytest.mark.gpu
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
@pytest.mark.parametrize("nx,k,nh", [(16, 3, 1), (40, 2, 2)])
def test_inner_loop_device_equals_host(ctx, precision, nx, k, nh):
    """The graph-resident inner PCG (device-side loop and stopping test)
    performs the host-driven loop's arithmetic in the same order: identical
    iteration counts and bit-identical solutions."""
    wl = synth.single_box_inclusion(nx, k, 1e4, n_hlevels=nh)
    eta, rho = materials.rasterise_inclusions(nx, nx, wl.shapes)
    prob, ref = pair(ctx, nx, nx, k, wl.bc, eta, nh=nh, seed=1, precision=precision)
    f = dev(sip.rhs_body_force(ref, rho))
    out = {}
    for mode in ["host", "device", "host"]:
        u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
        rep = prob.solve(f, u, p, rtol=1e-8, inner_loop=mode, inner_krylov="pcg",
                         inner_norm="true")
        out.setdefault(mode, []).append((rep, u, p))
    (rh, uh, ph), (rh2, uh2, ph2) = out["host"]
    rd, ud, pd_ = out["device"][0]
    assert torch.equal(uh, uh2) and torch.equal(ph, ph2)   # the solve is deterministic
    assert (rd["outer_its"], rd["inner_total"], rd["inner_max"]) == \
        (rh["outer_its"], rh["inner_total"], rh["inner_max"])
    assert torch.equal(ud, uh) and torch.equal(pd_, ph)
    assert rd["rel_residual"] == rh["rel_residual"] <= 1e-8



# ---- Q^2_0 coarse space (Sec. 6.1.1)
@pytest.mark.parametrize("nh,n,k,bc", [(2, 17, 2, SINK), (1, 9, 3, ("navier",) * 4),
                                       (0, 9, 2, ("dirichlet",) * 4)])
def test_q0_levels_and_vcycle(ctx, nh, n, k, bc):
    """Element-wise constant coarse space: the level-0 stencil equals the
    oracle's A_0 = P_0^T A P_0 on the element centres, the coarser levels its
    Galerkin products, the coarsest direct solve the dense solve, and one
    V-cycle the oracle's, to 1e-9."""
    eta, _ = materials.rasterise_inclusions(n, n, synth.single_box_inclusion(n, k, 1e3).shapes)
    prob, ref = pair(ctx, n, n, k, bc, eta, nh=nh, seed=6, coarse="q0")
    A = sip.assemble_A(ref)
    mg = multigrid.HPMultigrid(ref, A, nh, seed=6, coarse="q0")
    nl, nvx, nvy = prob.hlevel_dims(0)
    assert (nl, nvx, nvy) == (nh + 1, n, n)
    mats = [lv.A for lv in mg.h.levels] + [mg.h.coarse_A] if nh else [mg.A0.toarray()]
    for l in range(nh + 1):
        _, nvx, nvy = prob.hlevel_dims(l)
        x = synth.random_vector(2 * nvx * nvy, 40 + l)
        y = torch.empty_like(dev(x))
        prob.hlevel_apply(l, dev(x), y)
        assert rel(host(y), mats[l] @ x) < 1e-10, l
        if l < nh:
            assert abs(prob.lambda_max(l) - mg.h.levels[l].lmax) < 1e-9 * mg.h.levels[l].lmax
    _, nvx, nvy = prob.hlevel_dims(nh)
    b = synth.random_vector(2 * nvx * nvy, 7)
    x = torch.empty_like(dev(b))
    prob.coarse_solve(dev(b), x)
    assert rel(host(x), np.linalg.solve(np.asarray(mats[nh]), b)) < 1e-9
    assert abs(prob.lambda_max(-1) - mg.lmax) < 1e-9 * mg.lmax
    r = synth.random_vector(prob.n_u, 78)
    z = torch.empty_like(dev(r))
    prob.vcycle(dev(r), z)
    assert rel(host(z), mg(r)) < 1e-9
    prob.vcycle(dev(r), z)
    assert rel(host(z), mg(r)) < 1e-9


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_q0_box_inclusion(ctx, precision):
    """A_hp(Q^2_0): the box-inclusion Stokes problem on a 17 x 17 mesh (two
    cell-centred coarsenings) reaches the 1e-8 true residual and the
    sparse-direct solution."""
    n, k = 17, 2
    wl = synth.single_box_inclusion(n, k, 1e4, n_hlevels=2)
    eta, rho = materials.rasterise_inclusions(n, n, wl.shapes)
    prob, ref = pair(ctx, n, n, k, wl.bc, eta, nh=2, seed=1, precision=precision, coarse="q0")
    f = sip.rhs_body_force(ref, rho)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-8, max_outer=1000)
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.05e-8, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-5


def test_q0_rejects_even_meshes(ctx):
    """Cell-centred coarsening needs nx - 1 and ny - 1 divisible by 2^n_hlevels."""
    with pytest.raises(api.SipError):
        api.Problem(ctx, 16, 16, 2, np.ones(256), n_hlevels=1, coarse="q0")


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_solve_inner_preconditioned_norm(ctx, precision):
    """Inner solves stopped on the preconditioned residual ||V r|| (PETSc's
    default CG test): the Stokes solve still reaches the 1e-8 true residual
    and the sparse-direct solution, with fewer inner iterations than the
    residual test; in FP64 the iteration counts follow the oracle's FGMRES
    with the same inner test."""
    nx = ny = 16
    k = 3
    wl = synth.single_box_inclusion(nx, k, 1e4, n_hlevels=1)
    eta, rho = materials.rasterise_inclusions(nx, ny, wl.shapes)
    prob, ref = pair(ctx, nx, ny, k, wl.bc, eta, nh=1, seed=1, precision=precision)
    f = sip.rhs_body_force(ref, rho)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep_t = prob.solve(dev(f), u, p, rtol=1e-8, max_outer=1000, inner_norm="true")
    rep = prob.solve(dev(f), u, p, rtol=1e-8, max_outer=1000, inner_norm="preconditioned")
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.05e-8, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-5
    assert rep["inner_avg"] < rep_t["inner_avg"]
    if precision == "fp64":
        mg = multigrid.HPMultigrid(ref, A, 1, seed=1)
        pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(ref), mg, inner_norm="preconditioned")
        K = krylov.stokes_matrix(A, B).tocsr()
        b = np.concatenate([f, np.zeros(B.shape[1])])
        _, its, _ = krylov.fgmres(lambda v: K @ v, pc, b, 1e-8, restart=100, maxit=1000)
        assert abs(rep["outer_its"] - its) <= 1
        assert abs(rep["inner_avg"] - np.mean(pc.inner_its)) <= 0.5


@pytest.mark.parametrize("precision,restart", [("fp64", 30), ("fp64", 3), ("mixed", 30)])
def test_solve_inner_gcr(ctx, precision, restart):
    """Inner solves by restarted GCR (the method of the six-inclusion runs,
    Sec. 7.3), on the device loop: the Stokes solve reaches the 1e-8 true
    residual and the sparse-direct solution; in FP64 the outer and inner
    iteration counts follow the oracle's FGMRES with inner GCR of the same
    restart length."""
    nx = ny = 16
    k = 3
    wl = synth.single_box_inclusion(nx, k, 1e4, n_hlevels=1)
    eta, rho = materials.rasterise_inclusions(nx, ny, wl.shapes)
    prob, ref = pair(ctx, nx, ny, k, wl.bc, eta, nh=1, seed=1, precision=precision)
    f = sip.rhs_body_force(ref, rho)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-8, max_outer=1000, inner_krylov="gcr",
                     inner_restart=restart)
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.05e-8, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-5
    if restart == 3:
        assert rep["inner_max"] > 3, rep   # the restart was exercised
    if precision == "fp64":
        mg = multigrid.HPMultigrid(ref, A, 1, seed=1)
        pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(ref), mg, inner="gcr",
                                        inner_restart=restart)
        K = krylov.stokes_matrix(A, B).tocsr()
        b = np.concatenate([f, np.zeros(B.shape[1])])
        _, its, _ = krylov.fgmres(lambda v: K @ v, pc, b, 1e-8, restart=100, maxit=1000)
        assert abs(rep["outer_its"] - its) <= 1, (rep, its)
        assert abs(rep["inner_avg"] - np.mean(pc.inner_its)) <= 0.5, (rep, np.mean(pc.inner_its))


def test_gcr_options_rejected(ctx):
    """GCR runs on the device loop only, with 1 <= inner_restart <= 64."""
    nx = ny = 8
    eta = np.ones(nx * ny)
    prob = api.Problem(ctx, nx, ny, 2, eta, n_hlevels=1, seed=1)
    f = torch.ones(prob.n_u, dtype=torch.float64, device="cuda")
    u = torch.empty_like(f)
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    for kw in ({"inner_loop": "host", "inner_norm": "true"}, {"inner_restart": 0},
               {"inner_restart": 65}):
        with pytest.raises(api.SipError):
            prob.solve(f, u, p, inner_krylov="gcr", **kw)
    rep = prob.solve(f, u, p, inner_krylov="gcr", inner_restart=64)
    assert rep["status"] == 0


@pytest.mark.parametrize("inner", ["gcr", "pcg"])
def test_solve_outer_gcr(ctx, inner):
    """GCR as the outer method (the paper's choice for the six inclusions,
    Sec. 7.3): reaches the 1e-8 true residual and the sparse-direct
    solution, and its outer and inner iteration counts follow the oracle's
    outer GCR with the same inner method."""
    nx = ny = 16
    k = 3
    wl = synth.single_box_inclusion(nx, k, 1e4, n_hlevels=1)
    eta, rho = materials.rasterise_inclusions(nx, ny, wl.shapes)
    prob, ref = pair(ctx, nx, ny, k, wl.bc, eta, nh=1, seed=1)
    f = sip.rhs_body_force(ref, rho)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-8, max_outer=1000, outer_krylov="gcr",
                     inner_krylov=inner, inner_norm="true")
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.05e-8, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-5
    mg = multigrid.HPMultigrid(ref, A, 1, seed=1)
    pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(ref), mg, inner=inner)
    K = krylov.stokes_matrix(A, B).tocsr()
    b = np.concatenate([f, np.zeros(B.shape[1])])
    _, its = krylov.gcr_outer(lambda v: K @ v, pc, b, 1e-8, restart=100, maxit=1000)
    assert abs(rep["outer_its"] - its) <= 1, (rep, its)
    assert abs(rep["inner_avg"] - np.mean(pc.inner_its)) <= 0.5, (rep, np.mean(pc.inner_its))


def test_solve_outer_gcr_dirichlet_restarted(ctx):
    """Outer GCR restarted after 4 directions on the all-Dirichlet
    manufactured problem (constant pressure projected out): the sparse-direct
    solution to 1e-10 with a zero-mean pressure."""
    sol = exact.SmoothDirichlet()
    nx = ny = 8
    prob, ref = pair(ctx, nx, ny, 2, ("dirichlet",) * 4, np.ones(64), nh=0, seed=7)
    f = sip.rhs_force(ref, sol.f)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-10, restart=4, max_outer=400, outer_krylov="gcr",
                     inner_krylov="gcr")
    assert rep["outer_its"] > 4, rep
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.5e-10, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    assert rel(host(u), u_ref) < 1e-8
    assert abs(host(p)[::4].mean()) < 1e-12


@pytest.mark.parametrize("inner_norm", ["true", "preconditioned"])
def test_solve_checkerboard(ctx, inner_norm):
    """2 x 2 viscosity checkerboard 1e6 (Sec. 7.2) with a dense disc, Navier
    on every side (constant pressure projected out), A_hp(Q^2_1) with one
    h-coarsening: the 1e-8 true residual, the oracle FGMRES's outer and inner
    iteration counts with the same inner test, and a velocity as close to
    the sparse-direct one as the oracle's own iterate at the same residual
    (at this contrast a 1e-8 residual leaves ~1e-5 in u)."""
    n, k = 16, 2
    wl = synth.checkerboard(n=n, k=k, eta_hi=1e6, n_hlevels=1)
    eta, rho = materials.rasterise_inclusions(n, n, wl.shapes)
    prob, ref = pair(ctx, n, n, k, wl.bc, eta, nh=1, seed=1)
    f = sip.rhs_body_force(ref, rho)
    u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(dev(f), u, p, rtol=1e-8, max_outer=1000, inner_norm=inner_norm)
    res, A, B = _true_residual(ref, host(u), host(p), f)
    assert res <= 1.05e-8, rep
    u_ref, p_ref = krylov.solve_direct(ref, A, B, f)
    null = sip.pressure_constant(ref)
    mg = multigrid.HPMultigrid(ref, A, 1, seed=1)
    pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(ref), mg, null_p=null,
                                    inner_norm=inner_norm)
    K = krylov.stokes_matrix(A, B).tocsr()
    b = np.concatenate([f, np.zeros(B.shape[1])])
    x, its, _ = krylov.fgmres(lambda v: K @ v, pc, b, 1e-8, restart=100, maxit=1000,
                              null_p=null, n_u=A.shape[0])
    err_oracle = rel(x[:A.shape[0]], u_ref)
    assert rel(host(u), u_ref) < 4.0 * max(err_oracle, 1e-9), (rel(host(u), u_ref), err_oracle)
    assert abs(rep["outer_its"] - its) <= 1, (rep, its)
    assert abs(rep["inner_avg"] - np.mean(pc.inner_its)) <= 0.5, (rep, np.mean(pc.inner_its))
