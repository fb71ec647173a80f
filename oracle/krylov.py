"""Direct and Krylov solvers of the Stokes system (oracle).

Test infrastructure only (see ``oracle/__init__``).

* ``solve_direct``  sparse-direct solve of eq. discretestokes
  [A B; B^T 0][u; p] = [f; g], bordered by the constraint int p = 0 when
  there is no Neumann face (eq. pressure).
* ``pcg``           preconditioned CG on A with the relative stopping test
  ||A y - x|| / ||x|| < eps of Sec. 6 (inner viscous solve).
* ``gcr``           generalised conjugate residual, right-preconditioned,
  flexible, restarted: the Krylov method the paper ran for the viscous block
  of the six-inclusion problem (Sec. 7.3); stops on the residual itself.
* ``gcr_outer``     the same GCR as the outer Stokes solve with the block
  preconditioner (the paper's outer method for the six inclusions), with
  the true residual checked whenever the recurrence reports convergence.
* ``exact_residual`` / ``refine``  b - K x in exact rational arithmetic and
  iterative refinement of an FP64 solver with it (the precision question of
  Sec. 7.4, answered for the residual only).
* ``fgmres``        right-preconditioned flexible GMRES (Saad's FGMRES) on the
  saddle system with the upper block-triangular preconditioner of
  eq. discretestokespc, S replaced by the diagonal S* (Sec. 5), and
  A^{-1} replaced by an inner PCG solve (Sec. 6).  Stopping test: residual
  2-norm reduced by ``rtol`` from the initial one (Sec. 7 settings).
  Orthogonalisation: classical Gram-Schmidt applied twice.

Reading of the Schur block: the preconditioner's lower-right block is the
Schur complement of the saddle matrix itself, 0 - B^T A^{-1} B (negative
definite; the convention of the PETSc block factorisations the paper ran
with), approximated by -S*.  With exact blocks both signs give convergence
in two iterations (eigenvalue 1 with a 2x2 Jordan block for this sign,
+-1 for the other); with the inexact inner solve this sign reproduces the
paper's outer iteration counts and the other does not.
"""
from fractions import Fraction

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import sip


def stokes_matrix(A, B):
    return sp.bmat([[A, B], [B.T, None]], format="csr")


def solve_direct(prob, A, B, f, g=None):
    """Sparse-direct (SuperLU) solve of the saddle system.  Without a
    Neumann face the pressure is fixed by int_Omega p = 0."""
    n_u, n_p = B.shape
    g = np.zeros(n_p) if g is None else g
    K = stokes_matrix(A, B)
    rhs = np.concatenate([f, g])
    if not prob.has_neumann:
        w = sip.pressure_mass(prob) * sip.pressure_constant(prob)   # int psi_i
        col = sp.csr_matrix(np.concatenate([np.zeros(n_u), w])[:, None])
        K = sp.bmat([[K, col], [col.T, None]], format="csc")
        rhs = np.concatenate([rhs, [0.0]])
    sol = spla.spsolve(K.tocsc(), rhs)
    return sol[:n_u], sol[n_u:n_u + n_p]


def pcg(apply_A, precond, x, rtol, maxit=200, y0=None, norm="true"):
    """Preconditioned CG for A y = x.

    norm = "true": stops when ||A y - x|| < rtol ||x|| (the residual itself);
    norm = "preconditioned": stops when ||B r|| < rtol ||B r_0||, B the
    preconditioner, r = x - A y: the preconditioned residual that CG forms
    anyway for its next direction (the default test of PETSc's CG, which the
    paper ran).  The iterates are the same; only the stopping point differs.

    Returns (y, iterations)."""
    y = np.zeros_like(x) if y0 is None else y0.copy()
    r = x - apply_A(y) if y0 is not None else x.copy()
    nx = np.linalg.norm(x)
    if nx == 0.0:
        return y, 0
    z = precond(r)
    nz0 = np.linalg.norm(z)
    d = z.copy()
    rz = r @ z
    for it in range(1, maxit + 1):
        q = apply_A(d)
        alpha = rz / (d @ q)
        y += alpha * d
        r -= alpha * q
        if norm == "true" and np.linalg.norm(r) < rtol * nx:
            return y, it
        z = precond(r)
        if norm == "preconditioned" and np.linalg.norm(z) < rtol * nz0:
            return y, it
        rz_new = r @ z
        d = z + (rz_new / rz) * d
        rz = rz_new
    return y, maxit


def fcg(apply_A, precond, x, rtol, maxit=200, norm="true"):
    """Flexible conjugate gradients, FCG(1) (Notay, SIAM J. Sci. Comput. 22,
    2000), for A y = x from y = 0; stopping test as in ``pcg`` (``norm``).

    Each new direction is made A-orthogonal to the previous one explicitly,
    beta = <z, q_prev> / <d_prev, q_prev>, and the step is the exact line
    minimum along it, alpha = <d, r> / <d, q>.  With a fixed SPD
    preconditioner this is PCG; it stays convergent when the preconditioner
    varies a little between applications (a V-cycle in FP32).

    Returns (y, iterations)."""
    y = np.zeros_like(x)
    r = x.copy()
    nx = np.linalg.norm(x)
    if nx == 0.0:
        return y, 0
    z = precond(r)
    nz0 = np.linalg.norm(z)
    d = q = None
    for it in range(1, maxit + 1):
        if d is None:
            d = z.copy()
        else:
            d = z - (z @ q) / (d @ q) * d
        q = apply_A(d)
        alpha = (d @ r) / (d @ q)
        y += alpha * d
        r -= alpha * q
        if norm == "true" and np.linalg.norm(r) < rtol * nx:
            return y, it
        z = precond(r)
        if norm == "preconditioned" and np.linalg.norm(z) < rtol * nz0:
            return y, it
    return y, maxit


def gcr(apply_A, precond, x, rtol, maxit=200, norm="true", restart=30, on_z=None, proj=None):
    """Generalised conjugate residual method (Eisenstat, Elman & Schultz,
    SIAM J. Numer. Anal. 20, 1983) for A y = x from y = 0, preconditioned on
    the right, flexible (the preconditioner may change between steps) and
    restarted: the stored directions are dropped after ``restart`` of them.

    A step preconditions the residual, z = precond(r), and forms q = A z.
    It then orthogonalises q against the stored q_i and applies the same
    combination to z, so q = A z still holds: beta_i = <q, q_i> / <q_i, q_i>,
    q -= sum beta_i q_i, z -= sum beta_i z_i (classical Gram-Schmidt, done
    twice).  alpha = <r, q> / <q, q> then minimises ||r - alpha q||;
    y += alpha z, r -= alpha q, and (z, q) is stored.  Within a cycle y is
    the minimum-residual iterate over the span of the preconditioned
    residuals.  The test is ||x - A y|| < rtol ||x||, the quantity GCR
    minimises; ``norm`` must be "true".  ``on_z`` (tests) sees every
    preconditioned residual before orthogonalisation; ``proj`` (the Stokes
    solve without a Neumann side) is applied to z and to q = A z, keeping
    the constant pressure out of both (Sec. 5).

    Returns (y, iterations)."""
    if norm != "true":
        raise ValueError("GCR stops on the residual itself")
    y = np.zeros_like(x)
    r = x.copy()
    nx = np.linalg.norm(x)
    if nx == 0.0:
        return y, 0
    Zs, Qs, qq = [], [], []
    for it in range(1, maxit + 1):
        if len(Zs) == restart:
            Zs, Qs, qq = [], [], []
        z = precond(r)
        if proj is not None:
            z = proj(z)
        if on_z is not None:
            on_z(z.copy())
        q = apply_A(z)
        if proj is not None:
            q = proj(q)
        for _ in range(2):
            beta = [(q @ qi) / qqi for qi, qqi in zip(Qs, qq)]
            for b, zi, qi in zip(beta, Zs, Qs):
                q = q - b * qi
                z = z - b * zi
        qn = q @ q
        alpha = (r @ q) / qn
        y += alpha * z
        r -= alpha * q
        Zs.append(z)
        Qs.append(q)
        qq.append(qn)
        if np.linalg.norm(r) < rtol * nx:
            return y, it
    return y, maxit


class BlockPreconditioner:
    """Action of the upper block-triangular preconditioner inverse
    (eq. discretestokespc) with the Schur block -S* and A^{-1} -> an inner
    Krylov solve (PCG, FCG or GCR):
        y_p = -S*^{-1} x_p,   y_u ~= A^{-1} (x_u - B y_p)."""

    def __init__(self, A, B, s_diag, inner_precond, inner_rtol=1e-3,
                 inner_maxit=200, null_p=None, inner="pcg", inner_norm="true",
                 inner_restart=30):
        self.A, self.B, self.s = A, B, s_diag
        self.inner_kw = {"restart": inner_restart} if inner == "gcr" else {}
        self.inner_precond = inner_precond
        self.inner_rtol, self.inner_maxit = inner_rtol, inner_maxit
        self.null_p = null_p
        self.inner = {"pcg": pcg, "fcg": fcg, "gcr": gcr}[inner]
        self.inner_norm = inner_norm
        self.inner_its = []

    def __call__(self, x):
        n_u = self.A.shape[0]
        xu, xp = x[:n_u], x[n_u:]
        yp = -xp / self.s
        if self.null_p is not None:
            yp = project_out(yp, self.null_p)
        t = xu - self.B @ yp
        yu, its = self.inner(lambda v: self.A @ v, self.inner_precond, t,
                             self.inner_rtol, self.inner_maxit, norm=self.inner_norm,
                             **self.inner_kw)
        self.inner_its.append(its)
        return np.concatenate([yu, yp])


def project_out(v, z):
    return v - (z @ v) / (z @ z) * z


def fgmres(apply_K, precond, b, rtol, restart=100, maxit=200, null_p=None, n_u=None):
    """Right-preconditioned flexible GMRES (Saad, Alg. 9.6) with CGS2.

    Solves K x = b from x0 = 0; stops when ||b - K x||_2 <= rtol ||b||_2.
    ``null_p`` (with ``n_u``) projects the constant pressure out of every
    basis vector (Sec. 5, consistent right-hand side for a singular system).
    Returns (x, iterations, residual history)."""
    n = b.size
    x = np.zeros(n)
    beta0 = np.linalg.norm(b)
    hist = [beta0]
    if beta0 == 0.0:
        return x, 0, hist
    total = 0

    def proj(v):
        if null_p is None:
            return v
        v = v.copy()
        v[n_u:] = project_out(v[n_u:], null_p)
        return v

    r = proj(b.copy())
    while total < maxit:
        beta = np.linalg.norm(r)
        V = np.zeros((restart + 1, n))
        Z = np.zeros((restart, n))
        H = np.zeros((restart + 1, restart))
        V[0] = r / beta
        g = np.zeros(restart + 1)
        g[0] = beta
        cs = np.zeros(restart)
        sn = np.zeros(restart)
        j_done = 0
        for j in range(restart):
            Z[j] = proj(precond(V[j]))
            w = proj(apply_K(Z[j]))
            for _ in range(2):                      # classical Gram-Schmidt, twice
                h = V[:j + 1] @ w
                w = w - V[:j + 1].T @ h
                H[:j + 1, j] += h
            H[j + 1, j] = np.linalg.norm(w)
            if H[j + 1, j] > 0:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):                     # apply previous rotations
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = np.hypot(H[j, j], H[j + 1, j])
            cs[j], sn[j] = H[j, j] / den, H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            total += 1
            j_done = j + 1
            hist.append(abs(g[j + 1]))
            if abs(g[j + 1]) <= rtol * beta0 or total >= maxit:
                break
        yk = np.linalg.solve(np.triu(H[:j_done, :j_done]), g[:j_done])
        x = x + Z[:j_done].T @ yk
        r = proj(b - apply_K(x))
        if np.linalg.norm(r) <= rtol * beta0:
            break
    return x, total, hist


def gcr_outer(apply_K, precond, b, rtol, restart=100, maxit=200, null_p=None, n_u=None):
    """GCR (``gcr``) on the saddle system K x = b from x = 0 with the block
    preconditioner: stops when ||b - K x||_2 <= rtol ||b||_2 for the residual
    recomputed from x.  Each call of ``gcr`` solves for a correction of the
    current residual r = b - K x to the absolute level rtol ||b||; when the
    recurrence's residual meets it but the recomputed one does not, GCR
    starts again from the recomputed residual.  ``null_p`` as in ``fgmres``.
    Returns (x, iterations)."""
    x = np.zeros(b.size)
    nb = np.linalg.norm(b)
    if nb == 0.0:
        return x, 0

    def proj(v):
        if null_p is None:
            return v
        v = v.copy()
        v[n_u:] = project_out(v[n_u:], null_p)
        return v

    total = 0
    while total < maxit:
        r = proj(b - apply_K(x))
        nr = np.linalg.norm(r)
        if nr <= rtol * nb:
            break
        dx, its = gcr(apply_K, precond, r, rtol * nb / nr, maxit - total, restart=restart,
                      proj=proj if null_p is not None else None)
        x = x + dx
        total += its
    return x, total


def exact_residual(K, b, x):
    """b - K x evaluated exactly: K a scipy sparse matrix of FP64 entries, b
    FP64, x a sequence of exact rationals (``Fraction``); every FP64 number
    is a dyadic rational, so the result is the exact residual of the FP64
    matrix.  Returns a list of ``Fraction``."""
    K = K.tocsr()
    out = []
    for i in range(K.shape[0]):
        acc = Fraction(float(b[i]))
        for j in range(K.indptr[i], K.indptr[i + 1]):
            acc -= Fraction(float(K.data[j])) * x[K.indices[j]]
        out.append(acc)
    return out


def refine(K, solve, b, rtol, max_steps=10):
    """Iterative refinement: x accumulated exactly (rationals), r = b - K x
    exact (``exact_residual``), and each correction K d = r solved by the
    FP64 routine ``solve(r_fp64, rtol_step)`` asked for the reduction still
    missing, rtol_step = min(1/2, rtol ||b|| / ||r||).  Stops when
    ||r|| <= rtol ||b|| or when a step fails to halve ||r||.
    Returns (x as float64, list of exact relative residual norms)."""
    n = b.size
    x = [Fraction(0)] * n
    nb = float(np.linalg.norm(b))
    r = np.array(b, dtype=np.float64)
    nr = nb
    hist = []
    for _ in range(max_steps):
        d = solve(r, min(0.5, rtol * nb / nr))
        x = [xi + Fraction(float(di)) for xi, di in zip(x, d)]
        rx = exact_residual(K, b, x)
        r = np.array([float(v) for v in rx])
        nr_new = float(np.linalg.norm(r))
        hist.append(nr_new / nb)
        if nr_new <= rtol * nb or nr_new > 0.5 * nr:
            break
        nr = nr_new
    return np.array([float(v) for v in x]), hist
