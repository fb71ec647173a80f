"""Pins of the FP64 oracle against facts the paper and mathematics fix.

None of these re-derive the oracle's own formula: they use closed forms,
invariants, brute force, textbook values and convergence theory.
"""
import os

import numpy as np
import pytest

from oracle import basis, exact, krylov, materials, multigrid, rng, sip
from paper_1607_03777_gb300 import synth

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")
BCS = [("navier",) * 4, ("dirichlet",) * 4, ("navier", "navier", "navier", "neumann"),
       ("neumann", "dirichlet", "navier", "navier")]


def _prob(nx, ny, k, bc, seed=0, contrast=3.0, lx=1.0, ly=1.0):
    eta = 10.0 ** np.random.default_rng(seed).uniform(0, contrast, nx * ny)
    return sip.Problem(nx, ny, k, eta, bc=bc, lx=lx, ly=ly)


# ---------------------------------------------------------------- basis
def test_legendre_textbook_values():
    rows = np.loadtxt(os.path.join(GOLDEN, "legendre_orthonormal.txt"))
    for i, x, p in rows:
        val, _ = basis.legendre_values(int(i), np.array([x]))
        assert val[int(i), 0] == pytest.approx(np.sqrt((2 * i + 1) / 2) * p, rel=1e-14)


def test_legendre_orthonormal_by_dense_trapezoid():
    # brute-force integration on a fine grid (no Gauss rule involved)
    x = np.linspace(-1, 1, 200001)
    val, der = basis.legendre_values(6, x)
    M = np.trapezoid(val[:, None, :] * val[None, :, :], x, axis=2)
    assert np.abs(M - np.eye(7)).max() < 1e-8
    # derivative against central differences
    h = 1e-6
    vp, _ = basis.legendre_values(6, x[1000:1010] + h)
    vm, _ = basis.legendre_values(6, x[1000:1010] - h)
    assert np.abs((vp - vm) / (2 * h) - der[:, 1000:1010]).max() < 1e-6


# ---------------------------------------------------------------- rng
def test_splitmix64_published_vector():
    vals = [int(v) for v in np.loadtxt(os.path.join(GOLDEN, "splitmix64_seed1234567.txt"),
                                       dtype=np.uint64)]
    got = [int(v) for v in rng.splitmix64(1234567, 3)]
    assert got == vals


def test_uniform_range():
    u = rng.uniform_pm1(42, 100000)
    assert u.min() >= -1.0 and u.max() < 1.0 and abs(u.mean()) < 0.01


# ---------------------------------------------------------------- A
@pytest.mark.parametrize("bc", BCS)
@pytest.mark.parametrize("k", [1, 2, 3])
def test_A_symmetric_positive_definite(bc, k):
    """P1: A = A^T and A is SPD (SIP coercivity, Lemma 4.4)."""
    pr = _prob(3, 4, k, bc, seed=k)
    A = sip.assemble_A(pr).toarray()
    assert np.abs(A - A.T).max() <= 1e-14 * np.abs(A).max()
    np.linalg.cholesky(A)
    nb = pr.num.nb
    for e in range(pr.num.ne):     # element blocks SPD (M_K of Sec. 6)
        np.linalg.cholesky(A[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb])


@pytest.mark.parametrize("k", [1, 2, 4])
def test_A_closed_form_energies(k):
    """P2: on the unit square with Navier sides and constant eta,
    sigma_b = 8 eta (k+1)^2 / h: a((c,0),(c,0)) = 2 sigma_b c^2,
    a((x,0),(x,0)) = sigma_b - 2 eta, a((y,0),(y,0)) = eta + 2 sigma_b / 3."""
    nx, eta = 4, 1.7
    pr = sip.Problem(nx, nx, k, np.full(nx * nx, eta))
    A = sip.assemble_A(pr)
    sb = 8 * eta * (k + 1) ** 2 * nx
    cases = [(lambda x, y: (0.7 + 0 * x, 0 * x), 2 * sb * 0.49),
             (lambda x, y: (x, 0 * x), sb - 2 * eta),
             (lambda x, y: (y, 0 * x), eta + 2 * sb / 3),
             (lambda x, y: (0 * x, x), eta + 2 * sb / 3)]
    for f, expect in cases:
        u = sip.project_velocity(pr, f)
        assert u @ (A @ u) == pytest.approx(expect, rel=1e-12)


def test_A_rigid_rotation_energy_neumann():
    """A rigid rotation u = (-y, x) has eps(u) = 0 and no jumps, so with
    Neumann on every side its energy is exactly 0."""
    pr = sip.Problem(3, 3, 2, np.linspace(1, 5, 9), bc=("neumann",) * 4)
    A = sip.assemble_A(pr)
    u = sip.project_velocity(pr, lambda x, y: (-y, x))
    assert abs(u @ (A @ u)) < 1e-11 * np.abs(A).max()


def test_penalty_lower_bound_values():
    """Lemma 4.4 at its bound with tau = 0 and Lemma 4.1 on squares."""
    pr = sip.Problem(4, 4, 3, np.ones(16))
    assert sip.penalty(pr, 2.0, 5.0, 0.25) == pytest.approx(4 * 5.0 * 16 / 0.25)
    assert sip.penalty(pr, 2.0, None, 0.25) == pytest.approx(8 * 2.0 * 16 / 0.25)


def test_element_rows_match_assembly():
    pr = _prob(4, 3, 2, ("navier", "dirichlet", "neumann", "navier"))
    A = sip.assemble_A(pr).toarray()
    B = sip.assemble_B(pr).toarray()
    nb, mp = pr.num.nb, pr.num.mp
    for ex, ey in [(0, 0), (1, 1), (3, 2), (2, 0)]:
        e = pr.num.elem(ex, ey)
        row = np.zeros((nb, A.shape[1]))
        for f, blk in sip.element_rows_A(pr, ex, ey).items():
            row[:, f * nb:(f + 1) * nb] = blk
        assert np.abs(row - A[e * nb:(e + 1) * nb]).max() < 1e-12 * np.abs(A).max()
        rowb = np.zeros((nb, B.shape[1]))
        for f, blk in sip.element_rows_B(pr, ex, ey).items():
            rowb[:, f * mp:(f + 1) * mp] = blk
        assert np.abs(rowb - B[e * nb:(e + 1) * nb]).max() < 1e-13
        colb = np.zeros((mp, B.shape[0]))
        for f, blk in sip.element_cols_B(pr, ex, ey).items():
            colb[:, f * nb:(f + 1) * nb] = blk
        assert np.abs(colb - B.T[e * mp:(e + 1) * mp]).max() < 1e-13


# ---------------------------------------------------------------- B, S*
@pytest.mark.parametrize("k", [1, 2, 3])
def test_B_constant_pressure_null_space(k):
    """P3: without Neumann faces, b(u, 1) = 0 for every u, i.e. B 1 = 0;
    with a Neumann face the constant is not in the kernel."""
    pr = _prob(3, 3, k, ("navier", "dirichlet", "navier", "navier"))
    B = sip.assemble_B(pr)
    one = sip.pressure_constant(pr)
    assert np.abs(B @ one).max() < 1e-13
    pr2 = _prob(3, 3, k, ("navier", "navier", "navier", "neumann"))
    assert np.abs(sip.assemble_B(pr2) @ sip.pressure_constant(pr2)).max() > 1e-3


def test_B_divergence_of_linear_field():
    """b(u, q) for u = (x, 0) (div u = 1) on a Neumann box equals
    -int q (volume) + boundary-free jumps (u continuous) = -int q."""
    pr = sip.Problem(3, 2, 2, np.ones(6), bc=("neumann",) * 4)
    B = sip.assemble_B(pr)
    u = sip.project_velocity(pr, lambda x, y: (x, 0 * x))
    q = sip.project_pressure(pr, lambda x, y: 1 + x * y)
    # int_Omega (1 + x y) = 1 + 1/4
    assert u @ (B @ q) == pytest.approx(-(1 + 0.25), rel=1e-12)


def test_schur_mass_diagonal():
    """S* is diagonal for the orthonormal basis (Sec. 5): the full element
    pressure mass block equals (h_x h_y / 4) I."""
    pr = sip.Problem(2, 3, 4, np.ones(6), lx=1.0, ly=1.5)
    Mb = sip.pressure_mass_block(pr, 1, 2)
    assert np.abs(Mb - np.eye(16) * (0.5 * 0.5 / 4)).max() < 1e-15


# ---------------------------------------------------------------- exact solutions
@pytest.mark.parametrize("sol", [exact.SmoothNavier(2.0), exact.SmoothDirichlet(1.5),
                                 exact.PolynomialPatch()])
def test_exact_solutions_satisfy_pde(sol):
    """-div(2 eta eps(u)) + grad p = f and div u = 0 by finite differences."""
    eta = getattr(sol, "eta", 1.0)
    rng_ = np.random.default_rng(0)
    x, y = rng_.uniform(0.1, 0.9, 20), rng_.uniform(0.1, 0.9, 20)
    h = 1e-4

    def u(x_, y_):
        return np.array(sol.u(x_, y_))

    lap = (u(x + h, y) + u(x - h, y) + u(x, y + h) + u(x, y - h) - 4 * u(x, y)) / h ** 2
    gp = np.array([(sol.p(x + h, y) - sol.p(x - h, y)) / (2 * h),
                   (sol.p(x, y + h) - sol.p(x, y - h)) / (2 * h)])
    div = ((u(x + h, y) - u(x - h, y))[0] + (u(x, y + h) - u(x, y - h))[1]) / (2 * h)
    f = np.array(sol.f(x, y))
    assert np.abs(-eta * lap + gp - f).max() < 1e-4 * max(1, np.abs(f).max())
    assert np.abs(div).max() < 1e-6


# ---------------------------------------------------------------- discretisation
def _solve(sol, n, k, bc, eta=None):
    eta = np.full(n * n, getattr(sol, "eta", 1.0)) if eta is None else eta
    pr = sip.Problem(n, n, k, eta, bc=bc)
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    u, p = krylov.solve_direct(pr, A, B, sip.rhs_force(pr, sol.f))
    return pr, u, p


def test_patch_test_polynomial_solution_exact():
    """P4: u in Q_4^2, p in Q_3 with Dirichlet sides: SIP consistency makes
    the k = 4 discrete solution equal to the exact one."""
    sol = exact.PolynomialPatch()
    pr, u, p = _solve(sol, 3, 4, ("dirichlet",) * 4)
    eu, ep = sip.l2_errors(pr, u, p, sol.u, sol.p)
    assert eu < 1e-12 and ep < 1e-11


@pytest.mark.parametrize("k", [1, 2, 3])
def test_convergence_rates_smooth_navier(k):
    """P5: ||e_u|| ~ h^(k+1), ||e_p|| ~ h^k (a-priori estimates, Sec. 4.2;
    the paper's table shows 3.00 / 2.02 for k = 2)."""
    sol = exact.SmoothNavier(1.0)
    e = []
    for n in (4, 8):
        pr, u, p = _solve(sol, n, k, ("navier",) * 4)
        e.append(sip.l2_errors(pr, u, p, sol.u, sol.p))
    ru = np.log2(e[0][0] / e[1][0])
    rp = np.log2(e[0][1] / e[1][1])
    assert ru > k + 1 - 0.15
    assert rp > k - 0.15


@pytest.mark.parametrize("k", [1, 2])
def test_convergence_rates_viscosity_jump(k):
    """P5 with a mesh-aligned viscosity jump of 1e3 (pressure discontinuous)."""
    sol = exact.JumpNavier(1e3, 1.0, 0.25)
    e = []
    for n in (8, 16):
        pr = sip.Problem(n, n, k, sol.eta_elements(n, n))
        A, B = sip.assemble_A(pr), sip.assemble_B(pr)
        u, p = krylov.solve_direct(pr, A, B, sip.rhs_force(pr, sol.f))
        e.append(sip.l2_errors(pr, u, p, sol.u, sol.p))
    assert np.log2(e[0][0] / e[1][0]) > k + 1 - 0.15
    assert np.log2(e[0][1] / e[1][1]) > k - 0.15


def test_dirichlet_rates():
    sol = exact.SmoothDirichlet(1.0)
    e = []
    for n in (4, 8):
        pr, u, p = _solve(sol, n, 2, ("dirichlet",) * 4)
        e.append(sip.l2_errors(pr, u, p, sol.u, sol.p))
    assert np.log2(e[0][0] / e[1][0]) > 2.85


def test_body_force_load_vector():
    """f(v) for f = (0, -g rho): only the (0,0) mode of v_y sees it, with
    int phi_00 = |K| / 2 on the orthonormal basis."""
    pr = sip.Problem(2, 2, 2, np.ones(4))
    rho = np.array([1.0, 2.0, 3.0, 4.0])
    f = sip.rhs_body_force(pr, rho, g=10.0)
    F = f.reshape(4, 2, 3, 3)
    assert np.allclose(F[:, 1, 0, 0], -10 * rho * 0.25 / 2, rtol=1e-14)
    F[:, 1, 0, 0] = 0
    assert np.abs(F).max() < 1e-14


# ---------------------------------------------------------------- materials
def test_rasterise_brute_force():
    """eta = max over the open cell, rho = min over the cell, by dense
    point sampling of the cell (brute force)."""
    shapes = np.array([[0, 0.3, 0.4, 0.17, 0, 50.0, 1.5],
                       [0, 0.7, 0.7, 0.12, 0, 7.0, 1.2],
                       [1, 0.5, 0.77, 0.05, 0.31, 3.0, 1.1]])
    nx, ny = 12, 10
    eta, rho = materials.rasterise_inclusions(nx, ny, shapes)
    s = np.linspace(0, 1, 41)[1:-1]
    for e in range(nx * ny):
        ex, ey = e % nx, e // nx
        X, Y = np.meshgrid((ex + s) / nx, (ey + s) / ny)
        X, Y = X.ravel(), Y.ravel()
        et = np.ones_like(X)
        rh_in = []
        for kind, a, b, c, d, ei, ri in shapes:
            if kind == 0:
                ins = (X - a) ** 2 + (Y - b) ** 2 <= c ** 2
            else:
                ins = (X >= a) & (X <= b) & (Y >= c) & (Y <= d)
            et = np.where(ins, np.maximum(et, ei), et)
            rh_in.append(ri if ins.all() else 1.0)
        assert eta[e] == et.max(), e
        assert rho[e] == max(rh_in), e


def test_rasterise_mesh_aligned_box():
    eta, rho = materials.rasterise_inclusions(8, 8, [[1, 0.25, 0.75, 0.25, 0.75, 1e4, 1.2]])
    E = eta.reshape(8, 8)
    assert (E[2:6, 2:6] == 1e4).all() and E.sum() == 16 * 1e4 + 48


# ---------------------------------------------------------------- multigrid
def test_chebyshev_closed_form():
    """P8: on diag(lam) with M = I the Chebyshev error after m steps from
    x0 = 0 is T_m((theta - lam)/delta) / T_m(theta/delta) times the initial
    error (Chebyshev polynomial closed form)."""
    lam = np.linspace(0.2, 2.0, 30)
    b = np.ones(30)
    lo, hi = 0.1, 2.2
    th, de = (hi + lo) / 2, (hi - lo) / 2
    for m in (1, 2, 3, 5):
        x = multigrid.chebyshev(lambda v: lam * v, lambda v: v, b, None, m, lo, hi)
        err = x - b / lam
        T = np.polynomial.chebyshev.Chebyshev.basis(m)
        expect = T((th - lam) / de) / T(th / de) * (-b / lam)
        assert np.abs(err - expect).max() < 1e-13


def test_lambda_estimate_close_to_dense():
    """P10: 10 Arnoldi steps estimate lambda_max(M^{-1}A) within 5 %."""
    pr = _prob(6, 6, 2, ("navier", "navier", "navier", "neumann"), seed=3, contrast=2.0)
    A = sip.assemble_A(pr)
    blocks = multigrid.block_jacobi_blocks(A, pr.num.nb)
    inv = multigrid.invert_blocks(blocks)
    est = multigrid.estimate_lambda_max(lambda v: A @ v, lambda v: multigrid.block_apply(inv, v),
                                        A.shape[0], seed=11)
    Ad = A.toarray()
    Minv = np.zeros_like(Ad)
    nb = pr.num.nb
    for e in range(pr.num.ne):
        Minv[e * nb:(e + 1) * nb, e * nb:(e + 1) * nb] = inv[e]
    true = np.max(np.linalg.eigvals(Minv @ Ad).real)
    assert abs(est - true) / true < 0.05
    assert est <= true * (1 + 1e-10)


def test_galerkin_A1_is_order1_sip_with_fine_penalty():
    """P6: A_1 = P^T A P equals the order-1 SIP matrix assembled with the
    fine-degree trace constant (hierarchical basis, Sec. 6)."""
    pr = _prob(3, 3, 3, ("navier", "neumann", "dirichlet", "navier"), seed=5)
    A = sip.assemble_A(pr)
    P = multigrid.p_prolongation(3, pr.num.ne, 1)
    A1 = (P.T @ A @ P).toarray()
    pr1 = sip.Problem(3, 3, 1, pr.eta, bc=pr.bc, k_penalty=3)
    A1d = sip.assemble_A(pr1).toarray()
    assert np.abs(A1 - A1d).max() < 1e-12 * np.abs(A1).max()


def test_pcd_reproduces_bilinears():
    """P7: P_cd maps vertex values of a global bilinear to its exact modal
    Q_1 coefficients; P_h interpolates bilinears exactly."""
    nx, ny = 4, 3
    f = lambda x, y: (1 + 2 * x - y + 3 * x * y, -1 + x * y)
    vx, vy = np.meshgrid(np.arange(nx + 1) / nx, np.arange(ny + 1) / ny)
    fx, fy = f(vx.ravel(), vy.ravel())
    vert = np.stack([fx, fy], 1).ravel()
    Pcd = multigrid.continuous_to_dg(nx, ny)
    pr1 = sip.Problem(nx, ny, 1, np.ones(nx * ny))
    ref = sip.project_velocity(pr1, f)
    assert np.abs(Pcd @ vert - ref).max() < 1e-13
    P = multigrid.bilinear_prolongation(2, 3)
    cx, cy = np.meshgrid(np.arange(3) / 2, np.arange(4) / 3)
    fine_x, fine_y = np.meshgrid(np.arange(5) / 4, np.arange(7) / 6)
    g = lambda x, y: 2 - x + 4 * y + x * y
    coarse = np.stack([g(cx.ravel(), cy.ravel()), -g(cx.ravel(), cy.ravel())], 1).ravel()
    fine = np.stack([g(fine_x.ravel(), fine_y.ravel()), -g(fine_x.ravel(), fine_y.ravel())], 1).ravel()
    assert np.abs(P @ coarse - fine).max() < 1e-14


@pytest.mark.parametrize("nh", [0, 1])
def test_vcycle_symmetric(nh):
    """P11: the V-cycle is a symmetric operator, so PCG is legitimate."""
    pr = _prob(8, 8, 2, ("navier", "navier", "navier", "neumann"), seed=2, contrast=2.0)
    A = sip.assemble_A(pr)
    mg = multigrid.HPMultigrid(pr, A, nh, seed=9)
    g = np.random.default_rng(1)
    x, y = g.standard_normal(A.shape[0]), g.standard_normal(A.shape[0])
    assert abs(mg(x) @ y - x @ mg(y)) < 1e-11 * abs(x @ mg(y))


@pytest.mark.parametrize("sign", [-1.0, 1.0])
def test_exact_block_preconditioner_two_iterations(sign):
    """P9: with exact A^{-1} and the exact Schur complement (either sign:
    -B^T A^{-1} B, the saddle matrix's own Schur complement, or +B^T A^{-1} B)
    the upper block triangular preconditioner converges in at most 2
    iterations (Sec. 5)."""
    pr = _prob(3, 3, 2, ("navier", "navier", "navier", "neumann"), seed=4)
    A, B = sip.assemble_A(pr).toarray(), sip.assemble_B(pr).toarray()
    Ainv = np.linalg.inv(A)
    S = B.T @ Ainv @ B
    Sinv = np.linalg.inv(sign * S)
    n_u = A.shape[0]
    K = np.block([[A, B], [B.T, np.zeros((B.shape[1],) * 2)]])
    b = np.random.default_rng(0).standard_normal(K.shape[0])

    def prec(x):
        yp = Sinv @ x[n_u:]
        return np.concatenate([Ainv @ (x[:n_u] - B @ yp), yp])

    x, its, hist = krylov.fgmres(lambda v: K @ v, prec, b, 1e-10)
    assert its <= 3
    assert np.linalg.norm(b - K @ x) <= 1e-9 * np.linalg.norm(b)


def test_fgmres_hpmg_solves_to_direct_solution():
    """The oracle's block-preconditioned FGMRES with the two-level A_p(Q_1)
    preconditioner reaches the sparse-direct solution (config 1 shape)."""
    sol = exact.SmoothDirichlet()
    pr = sip.Problem(8, 8, 2, np.ones(64), bc=("dirichlet",) * 4)
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    f = sip.rhs_force(pr, sol.f)
    mg = multigrid.HPMultigrid(pr, A, 0, seed=7)
    null = sip.pressure_constant(pr)
    Pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(pr), mg, 1e-3, null_p=null)
    K = krylov.stokes_matrix(A, B)
    b = np.concatenate([f, np.zeros(B.shape[1])])
    x, its, _ = krylov.fgmres(lambda v: K @ v, Pc, b, 1e-10, null_p=null, n_u=A.shape[0])
    u, p = krylov.solve_direct(pr, A, B, f)
    assert its <= 30
    assert np.linalg.norm(b - K @ x) <= 1e-10 * np.linalg.norm(b) * 1.01
    assert np.linalg.norm(x[:A.shape[0]] - u) <= 1e-8 * np.linalg.norm(u)


def test_block_preconditioner_uses_negative_schur_block():
    """The oracle's preconditioner applies y_p = -S*^{-1} x_p, and with the
    inexact inner solve the outer count on a viscosity-jump problem stays in
    the paper's range (SolCx k = 2, Delta eta = 1e6: 5 outer iterations; the
    manufactured analogue here needs <= 12)."""
    sol = exact.JumpNavier(1e6, 1.0, 0.5)
    n = 16
    pr = sip.Problem(n, n, 2, sol.eta_elements(n, n))
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    s = sip.schur_mass(pr)
    mg = multigrid.HPMultigrid(pr, A, 1, seed=7)
    null = sip.pressure_constant(pr)
    Pc = krylov.BlockPreconditioner(A, B, s, mg, 1e-3, null_p=null)
    x = np.zeros(A.shape[0] + B.shape[1])
    x[A.shape[0]:] = s
    y = Pc(x)
    assert np.allclose(krylov.project_out(-np.ones(B.shape[1]), null), y[A.shape[0]:])
    K = krylov.stokes_matrix(A, B)
    b = np.concatenate([sip.rhs_force(pr, sol.f), np.zeros(B.shape[1])])
    _, its, _ = krylov.fgmres(lambda v: K @ v, Pc, b, 1e-6, null_p=null, n_u=A.shape[0])
    assert its <= 12


def _spd(n, seed, cond=1e4):
    g = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(g.standard_normal((n, n)))
    ev = np.logspace(0, np.log10(cond), n)
    return (Q * ev) @ Q.T


def test_fcg_equals_pcg_with_fixed_preconditioner():
    """FCG(1) and PCG coincide in exact arithmetic for a fixed SPD
    preconditioner (the explicit A-orthogonalisation reproduces PCG's beta):
    same iteration count, iterates equal to rounding."""
    A = _spd(40, 1, cond=1e2)
    dinv = 1.0 / np.diag(A)
    x = np.random.default_rng(2).standard_normal(40)
    for m in (1, 3, 8):   # iterates after m steps (before rounding drift)
        y1, i1 = krylov.pcg(lambda v: A @ v, lambda r: dinv * r, x, 1e-14, maxit=m)
        y2, i2 = krylov.fcg(lambda v: A @ v, lambda r: dinv * r, x, 1e-14, maxit=m)
        assert i1 == i2 == m
        assert np.linalg.norm(y1 - y2) <= 1e-10 * np.linalg.norm(y1)
    y1, i1 = krylov.pcg(lambda v: A @ v, lambda r: dinv * r, x, 1e-10, maxit=400)
    y2, i2 = krylov.fcg(lambda v: A @ v, lambda r: dinv * r, x, 1e-10, maxit=400)
    assert abs(i1 - i2) <= 1
    assert np.linalg.norm(A @ y2 - x) < 1e-10 * np.linalg.norm(x)


def test_fcg_exact_preconditioner_one_step():
    """With B = A^{-1} the first direction is the exact error: one iteration."""
    A = _spd(25, 3, cond=1e3)
    Ainv = np.linalg.inv(A)
    x = np.random.default_rng(4).standard_normal(25)
    y, its = krylov.fcg(lambda v: A @ v, lambda r: Ainv @ r, x, 1e-9)
    assert its == 1
    assert np.linalg.norm(A @ y - x) < 1e-9 * np.linalg.norm(x)


def test_fcg_tolerates_varying_preconditioner():
    """A preconditioner perturbed by a fresh 5% random diagonal at every
    application (not a fixed linear operator): FCG(1) still converges to
    1e-8 within a modest iteration count."""
    A = _spd(60, 5, cond=1e3)
    dinv = 1.0 / np.diag(A)
    g = np.random.default_rng(6)
    x = g.standard_normal(60)
    prec = lambda r: dinv * r * (1.0 + 0.05 * g.standard_normal(60))
    y, its = krylov.fcg(lambda v: A @ v, prec, x, 1e-8, maxit=500)
    assert np.linalg.norm(A @ y - x) < 1e-8 * np.linalg.norm(x)
    assert its < 300


def _parity_classes(k):
    n = k + 1
    out = []
    for c in range(2):
        for j in range(n):
            for i in range(n):
                out.append(((i + (c == 0)) & 1) | (((j + (c == 1)) & 1) << 1))
    return np.array(out)


@pytest.mark.parametrize("k", [1, 2, 3])
def test_element_block_reflection_parity(k):
    """The diagonal block of an element whose opposite faces are alike
    (interior with equal penalties, or boundary of one kind) couples only
    velocity modes of equal reflection parity, (-1)^(i + [c = x]) in x and
    (-1)^(j + [c = y]) in y; an element with one boundary x-face and one
    interior x-face couples the x-parities."""
    nx = ny = 3
    prob = sip.Problem(nx, ny, k, np.ones(nx * ny), bc=("navier",) * 4)
    A = sip.assemble_A(prob).tocsr()
    nb = prob.num.nb
    blocks = multigrid.block_jacobi_blocks(A, nb)
    par = _parity_classes(k)
    same_x = (par[:, None] & 1) == (par[None, :] & 1)
    same_y = (par[:, None] & 2) == (par[None, :] & 2)
    centre = blocks[4]                       # all four faces interior
    scale = np.abs(centre).max()
    assert np.abs(centre[~(same_x & same_y)]).max() <= 1e-13 * scale
    corner = blocks[0]                       # Navier left and bottom, interior right and top
    assert np.abs(corner[~same_x]).max() > 1e-3 * np.abs(corner).max()
    strip = sip.Problem(1, 3, k, np.ones(3), bc=("navier",) * 4)   # both x-faces Navier
    Bs = multigrid.block_jacobi_blocks(sip.assemble_A(strip).tocsr(), nb)
    mid = Bs[1]                              # x: Navier both sides; y: interior both sides
    assert np.abs(mid[~(same_x & same_y)]).max() <= 1e-13 * np.abs(mid).max()
    # the inverse keeps the structure
    inv = np.linalg.inv(centre)
    assert np.abs(inv[~(same_x & same_y)]).max() <= 1e-12 * np.abs(inv).max()


def _q0_closed_form(nx, ny, k, eta, bc, lx, ly):
    """The SIP form restricted to element-wise constants, written out: on a
    constant the strain vanishes, so only the penalty terms remain.  The
    constant mode is l_0(x) l_0(y) = 1/2 on the reference square, so a face
    of length h_t contributes sigma h_t / 4 per pair of traces;
    sigma = 4 max(eta) (k+1)^2 / h_n inside, 8 eta_K (k+1)^2 / h_n on a
    Navier (normal component) or Dirichlet (both components) side."""
    hx, hy = lx / nx, ly / ny
    n = 2 * nx * ny
    A = np.zeros((n, n))
    kk = (k + 1) ** 2
    for ey in range(ny):
        for ex in range(nx):
            e = ey * nx + ex
            for d, (hn, ht) in enumerate([(hx, hy), (hy, hx)]):
                for side in (0, 1):
                    nxe = ex + (side * 2 - 1 if d == 0 else 0)
                    nye = ey + (side * 2 - 1 if d == 1 else 0)
                    if 0 <= nxe < nx and 0 <= nye < ny:
                        if side == 0:
                            continue            # each interior face once, from its left/bottom side
                        f = nye * nx + nxe
                        w = 4.0 * max(eta[e], eta[f]) * kk / hn * ht / 4.0
                        for c in range(2):
                            A[2 * e + c, 2 * e + c] += w
                            A[2 * f + c, 2 * f + c] += w
                            A[2 * e + c, 2 * f + c] -= w
                            A[2 * f + c, 2 * e + c] -= w
                    else:
                        kind = bc[2 * d + side]
                        w = 8.0 * eta[e] * kk / hn * ht / 4.0
                        comps = {"navier": [d], "dirichlet": [0, 1], "neumann": []}[kind]
                        for c in comps:
                            A[2 * e + c, 2 * e + c] += w
    return A


@pytest.mark.parametrize("k", [1, 2, 4])
def test_q0_galerkin_operator_closed_form(k):
    """A_0 = P_0^T A P_0 (the element-wise constant coarse space, Sec. 6.1.1)
    equals the penalty-only 5-point operator written out independently, on a
    non-square mesh with random viscosity and Navier, Neumann and Dirichlet
    sides."""
    nx, ny, lx, ly = 3, 5, 1.5, 1.0
    eta = 10.0 ** np.random.default_rng(11).uniform(0, 2, nx * ny)
    bc = ("navier", "dirichlet", "neumann", "navier")
    prob = sip.Problem(nx, ny, k, eta, bc=bc, lx=lx, ly=ly)
    A = sip.assemble_A(prob).tocsr()
    P0 = multigrid.p_prolongation(k, nx * ny, 0)
    A0 = (P0.T @ A @ P0).toarray()
    ref = _q0_closed_form(nx, ny, k, eta, bc, lx, ly)
    assert np.abs(A0 - ref).max() <= 1e-12 * np.abs(ref).max()


@pytest.mark.parametrize("nh", [0, 2])
def test_q0_vcycle_symmetric_and_convergent(nh):
    """The hp-multigrid cycle with the Q^2_0 coarse space (A_p(Q^2_0) with an
    exact coarse solve, A_hp(Q^2_0) with two cell-centred coarsenings of a
    9 x 9 mesh) is a symmetric operator and makes PCG converge."""
    n, k = 9, 2
    eta = 10.0 ** np.random.default_rng(12).uniform(0, 2, n * n)
    prob = sip.Problem(n, n, k, eta, bc=("navier", "navier", "navier", "neumann"))
    A = sip.assemble_A(prob).tocsr()
    mg = multigrid.HPMultigrid(prob, A, nh, seed=3, coarse="q0")
    g = np.random.default_rng(13)
    x, y = g.standard_normal(A.shape[0]), g.standard_normal(A.shape[0])
    a, b = x @ mg(y), mg(x) @ y
    assert abs(a - b) <= 1e-11 * (abs(a) + abs(b))
    rhs = g.standard_normal(A.shape[0])
    sol, its = krylov.pcg(lambda v: A @ v, mg, rhs, 1e-8, maxit=200)
    assert np.linalg.norm(A @ sol - rhs) < 1e-8 * np.linalg.norm(rhs)
    assert its < 120


@pytest.mark.parametrize("solver", ["pcg", "fcg"])
def test_inner_preconditioned_norm_stopping(solver):
    """The preconditioned-residual stopping test (||B r|| < rtol ||B r_0||, B
    the preconditioner) changes only where CG stops: the iterate is the one
    the true-residual variant has after the same number of steps, the test
    holds there, and it did not hold one step earlier."""
    A = _spd(50, 21, cond=1e3)
    dinv = 1.0 / np.diag(A)
    x = np.random.default_rng(22).standard_normal(50)
    f = getattr(krylov, solver)
    B = lambda r: dinv * r
    y, its = f(lambda v: A @ v, B, x, 1e-4, maxit=400, norm="preconditioned")
    assert 1 < its < 400
    assert np.linalg.norm(B(x - A @ y)) < 1e-4 * np.linalg.norm(B(x))
    y2, its2 = f(lambda v: A @ v, B, x, 1e-30, maxit=its, norm="true")
    assert its2 == its and np.linalg.norm(y2 - y) <= 1e-12 * np.linalg.norm(y)
    y3, _ = f(lambda v: A @ v, B, x, 1e-30, maxit=its - 1, norm="true")
    assert not np.linalg.norm(B(x - A @ y3)) < 1e-4 * np.linalg.norm(B(x))


def _nonsym(n, seed):
    g = np.random.default_rng(seed)
    return 4.0 * np.eye(n) + g.standard_normal((n, n)) / np.sqrt(n)


def _min_residual_update(A, r0, Y):
    """argmin over y in span(Y) of ||r0 - A y|| by dense least squares."""
    c, *_ = np.linalg.lstsq(A @ Y, r0, rcond=None)
    return Y @ c


def _right_krylov(A, M, r0, j):
    """Columns spanning M K_j(A M, r0), built from an orthonormal basis of
    the Krylov space (modified Gram-Schmidt, so that the columns stay well
    conditioned)."""
    V = np.zeros((r0.size, j))
    v = r0 / np.linalg.norm(r0)
    for i in range(j):
        V[:, i] = v
        w = A @ (M @ v)
        for l in range(i + 1):
            w = w - (V[:, l] @ w) * V[:, l]
        v = w / np.linalg.norm(w)
    return M @ V


def test_gcr_is_minimum_residual_over_right_krylov_space():
    """With a fixed preconditioner M and no restart, GCR's j-th iterate is
    the minimiser of ||x - A y|| over y in M K_j(A M, x) (its defining
    property; Eisenstat, Elman & Schultz 1983), here computed by dense least
    squares on an explicit Krylov basis, for a nonsymmetric A."""
    n = 30
    A = _nonsym(n, 31)
    g = np.random.default_rng(32)
    M = np.diag(0.5 + g.random(n)) + 0.05 * g.standard_normal((n, n))
    x = g.standard_normal(n)
    for j in (1, 2, 5, 9):
        y, its = krylov.gcr(lambda v: A @ v, lambda r: M @ r, x, 0.0, maxit=j, restart=50)
        assert its == j
        ye = _min_residual_update(A, x, _right_krylov(A, M, x, j))
        assert np.linalg.norm(y - ye) <= 1e-10 * np.linalg.norm(ye)
        assert abs(np.linalg.norm(x - A @ y) - np.linalg.norm(x - A @ ye)) <= 1e-12 * np.linalg.norm(x)


def test_gcr_restart_minimises_per_cycle():
    """Restarted after m directions, GCR(m) is a sequence of minimum-residual
    corrections, each over the right Krylov space of the residual left by
    the previous cycle (cycles of 3, 3 and 1 steps for 7 iterations)."""
    n = 24
    A = _nonsym(n, 33)
    M = np.diag(np.random.default_rng(34).random(n) + 0.5)
    x = np.random.default_rng(35).standard_normal(n)
    y, its = krylov.gcr(lambda v: A @ v, lambda r: M @ r, x, 0.0, maxit=7, restart=3)
    assert its == 7
    ye = np.zeros(n)
    for j in (3, 3, 1):
        r = x - A @ ye
        ye = ye + _min_residual_update(A, r, _right_krylov(A, M, r, j))
    assert np.linalg.norm(y - ye) <= 1e-10 * np.linalg.norm(ye)


def test_gcr_flexible_minimises_over_preconditioned_residuals():
    """With a preconditioner that changes at every application, the iterate
    minimises the residual over the span of the vectors the preconditioner
    returned (the flexible property the outer and inner solves rely on)."""
    n = 28
    A = _nonsym(n, 36)
    g = np.random.default_rng(37)
    x = g.standard_normal(n)
    prec = lambda r: (0.5 + g.random(n)) * r
    zs = []
    y, its = krylov.gcr(lambda v: A @ v, prec, x, 0.0, maxit=6, restart=50, on_z=zs.append)
    assert its == 6 and len(zs) == 6
    ye = _min_residual_update(A, x, np.array(zs).T)
    assert np.linalg.norm(y - ye) <= 1e-10 * np.linalg.norm(ye)


def test_gcr_stops_at_first_step_below_tolerance():
    """GCR stops at the first step whose residual is below rtol ||x||; the
    minimum residual one step earlier is not."""
    n = 40
    A = _nonsym(n, 38)
    M = np.diag(1.0 / np.diag(A))
    x = np.random.default_rng(39).standard_normal(n)
    rtol = 1e-7
    y, its = krylov.gcr(lambda v: A @ v, lambda r: M @ r, x, rtol, maxit=100, restart=100)
    assert 1 < its < 100
    assert np.linalg.norm(x - A @ y) < rtol * np.linalg.norm(x)
    yp = _min_residual_update(A, x, _right_krylov(A, M, x, its - 1))
    assert not np.linalg.norm(x - A @ yp) < rtol * np.linalg.norm(x)
    with pytest.raises(ValueError):
        krylov.gcr(lambda v: A @ v, lambda r: M @ r, x, rtol, norm="preconditioned")


def test_gcr_hpmg_residual_monotone():
    """GCR preconditioned by the hp-multigrid V-cycle on a heterogeneous SIP
    viscous block: the residual norm never increases from one step to the
    next (minimum-residual property) and reaches the inner tolerance."""
    eta, _ = materials.rasterise_box(8, 8, (0.25, 0.75, 0.25, 0.75), 1e4, 1.0)
    prob = sip.Problem(8, 8, 2, eta, bc=("navier", "navier", "navier", "neumann"))
    A = sip.assemble_A(prob).tocsr()
    mg = multigrid.HPMultigrid(prob, A, 1, seed=3)
    x = np.random.default_rng(40).standard_normal(A.shape[0])
    res = []
    for j in range(1, 9):
        y, _ = krylov.gcr(lambda v: A @ v, mg, x, 0.0, maxit=j)
        res.append(np.linalg.norm(x - A @ y))
    assert all(b <= a * (1 + 1e-12) for a, b in zip(res, res[1:]))
    y, its = krylov.gcr(lambda v: A @ v, mg, x, 1e-3)
    assert its < 30 and np.linalg.norm(x - A @ y) < 1e-3 * np.linalg.norm(x)


@pytest.mark.parametrize("sign", [-1.0, 1.0])
def test_gcr_outer_exact_block_preconditioner_two_iterations(sign):
    """The outer GCR with the exact block preconditioner (either Schur sign)
    converges in at most 2 iterations, like FGMRES: the preconditioned
    saddle operator has a minimal polynomial of degree 2 (Sec. 5), and GCR
    minimises the residual over the same space for a fixed preconditioner."""
    pr = _prob(3, 3, 2, ("navier", "navier", "navier", "neumann"), seed=4)
    A, B = sip.assemble_A(pr).toarray(), sip.assemble_B(pr).toarray()
    Ainv = np.linalg.inv(A)
    Sinv = np.linalg.inv(sign * (B.T @ Ainv @ B))
    n_u = A.shape[0]
    K = np.block([[A, B], [B.T, np.zeros((B.shape[1],) * 2)]])
    b = np.random.default_rng(0).standard_normal(K.shape[0])

    def prec(x):
        yp = Sinv @ x[n_u:]
        return np.concatenate([Ainv @ (x[:n_u] - B @ yp), yp])

    x, its = krylov.gcr_outer(lambda v: K @ v, prec, b, 1e-10)
    assert its <= 3
    assert np.linalg.norm(b - K @ x) <= 1e-9 * np.linalg.norm(b)


def test_gcr_outer_hpmg_singular_pressure_solves_to_direct_solution():
    """GCR outer and inner with the hp-multigrid V-cycle on an all-Dirichlet
    problem (constant pressure in the null space, projected out): reaches
    the sparse-direct solution, and the iteration count is that of FGMRES
    with the same preconditioner to within two (both minimise the residual;
    the spaces differ only through the inexact inner solve)."""
    sol = exact.SmoothDirichlet()
    pr = sip.Problem(8, 8, 2, np.ones(64), bc=("dirichlet",) * 4)
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    f = sip.rhs_force(pr, sol.f)
    mg = multigrid.HPMultigrid(pr, A, 1, seed=7)
    null = sip.pressure_constant(pr)
    K = krylov.stokes_matrix(A, B)
    b = np.concatenate([f, np.zeros(B.shape[1])])
    n_u = A.shape[0]
    Pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(pr), mg, 1e-3, null_p=null, inner="gcr")
    x, its = krylov.gcr_outer(lambda v: K @ v, Pc, b, 1e-10, null_p=null, n_u=n_u)
    Pf = krylov.BlockPreconditioner(A, B, sip.schur_mass(pr), mg, 1e-3, null_p=null, inner="gcr")
    _, its_f, _ = krylov.fgmres(lambda v: K @ v, Pf, b, 1e-10, null_p=null, n_u=n_u)
    u, p = krylov.solve_direct(pr, A, B, f)
    assert abs(its - its_f) <= 2, (its, its_f)
    assert np.linalg.norm(b - K @ x) <= 1e-10 * np.linalg.norm(b)
    assert np.linalg.norm(x[:n_u] - u) <= 1e-8 * np.linalg.norm(u)
    assert abs(null @ x[n_u:]) <= 1e-10 * np.linalg.norm(x[n_u:]) * np.linalg.norm(null)


def test_exact_residual_matches_fp64_residual():
    """The exact rational residual agrees with the FP64 one to FP64 rounding
    (plumbing check against an independent evaluation)."""
    pr = _prob(3, 3, 2, ("navier", "navier", "navier", "neumann"), seed=5)
    A, B = sip.assemble_A(pr), sip.assemble_B(pr)
    K = krylov.stokes_matrix(A, B).tocsr()
    g = np.random.default_rng(41)
    b, x = g.standard_normal(K.shape[0]), g.standard_normal(K.shape[0])
    from fractions import Fraction
    r = np.array([float(v) for v in krylov.exact_residual(K, b, [Fraction(float(v)) for v in x])])
    assert np.linalg.norm(r - (b - K @ x)) <= 1e-13 * np.linalg.norm(b - K @ x)


def test_refine_reaches_below_fp64_floor():
    """Six inclusions, contrast 1e8, 16^2, k = 2: the FP64 FGMRES stalls with
    an exact residual near 3e-8 (no FP64 vector does much better: the
    rounding of the refined iterate sits at the same floor), while
    refinement with the exact residual takes the iterate below 1e-11 in one
    cheap correction (Sec. 7.4's precision question, for the residual)."""
    from fractions import Fraction
    n, k = 16, 2
    wl = synth.six_sinkers(n=n, k=k, eta_in=1e8, n_hlevels=1)
    eta, rho = materials.rasterise_inclusions(n, n, wl.shapes)
    pr = sip.Problem(n, n, k, eta, bc=wl.bc)
    A, B = sip.assemble_A(pr).tocsr(), sip.assemble_B(pr).tocsr()
    mg = multigrid.HPMultigrid(pr, A, 1, seed=1)
    f = sip.rhs_body_force(pr, rho, 10.0)
    K = krylov.stokes_matrix(A, B).tocsr()
    b = np.concatenate([f, np.zeros(B.shape[1])])

    def solve(r, rt):
        pc = krylov.BlockPreconditioner(A, B, sip.schur_mass(pr), mg, 1e-3)
        return krylov.fgmres(lambda v: K @ v, pc, r, rt, restart=100, maxit=60)[0]

    x64 = solve(b, 1e-12)
    nb = np.linalg.norm(b)
    exact_rel = lambda x: np.linalg.norm(
        [float(v) for v in krylov.exact_residual(K, b, [Fraction(float(t)) for t in x])]) / nb
    plain = exact_rel(x64)
    assert plain > 1e-9
    x_ir, hist = krylov.refine(K, solve, b, 1e-11, max_steps=4)
    assert hist[-1] <= 1e-11 and len(hist) <= 3, hist
    assert exact_rel(x_ir) > 100 * hist[-1]   # the FP64 rounding is back at the floor


def test_checkerboard_rasterised_quadrants():
    """The checkerboard input: eta_hi exactly on the elements of the lower-
    left and upper-right quadrants, 1 elsewhere (the jumps lie on element
    faces for even meshes); density 1.2 only on elements wholly inside the
    driving disc, which lies in the upper-left quadrant; Navier sides."""
    n = 16
    wl = synth.checkerboard(n=n, k=2, eta_hi=1e6, n_hlevels=2)
    eta, rho = materials.rasterise_inclusions(n, n, wl.shapes)
    xc = (np.arange(n) + 0.5) / n
    X, Y = np.meshgrid(xc, xc)            # element centres, row-major (ey, ex)
    hi = (X < 0.5) == (Y < 0.5)
    assert np.array_equal(eta.reshape(n, n), np.where(hi, 1e6, 1.0))
    dense = rho.reshape(n, n) > 1.0
    assert dense.any() and np.all(rho.reshape(n, n)[dense] == 1.2)
    assert np.all((X[dense] < 0.5) & (Y[dense] > 0.5))
    assert np.all((X[dense] - 0.3) ** 2 + (Y[dense] - 0.65) ** 2 < 0.1 ** 2)
    assert wl.bc == ("navier",) * 4
