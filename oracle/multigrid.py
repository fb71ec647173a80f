"""hp-multigrid preconditioner for the viscous block (oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. 6 of the paper, built from explicitly assembled matrices:

* two-level p-multigrid (Algorithm 1, one cycle per application) with
  aggressive coarsening Q_k -> Q_1 (or Q_0) in one step; prolongation is the
  injection of the hierarchical modes, restriction its transpose, and the
  coarse operator the Galerkin product A_s = P^T A P;
* smoother: Chebyshev iteration preconditioned by element-block Jacobi
  (the diagonal blocks of A), bounds [0.1 lam*, 1.1 lam*] with lam* the
  largest Ritz value of 10 GMRES (Arnoldi) steps on M^{-1}A started from a
  random vector;
* Q^2_1 coarse problem (Sec. 6.1.2): continuous bilinears via
  P_cd (element-wise nodal -> modal), A_1c = P_cd^T A_1 P_cd, a vertex-centred
  hierarchy with bilinear P_h and R_h = P_h^T, Galerkin coarse operators,
  Chebyshev / point-Jacobi smoothing and LU on the coarsest level;
* A_p(Q^2_1) variant (no h-levels): the coarse problem A_1 is solved by LU.

Readings where the paper is silent: the Chebyshev recurrence is the
classical one for SPD operators (Saad, Iterative Methods for Sparse Linear
Systems, Sec. 12.3, with M^{-1} applied to every residual); "m steps" means m
updates of the iterate; the eigen estimate runs on the preconditioned
operator, starting from M^{-1} b with b a SplitMix64 vector; the eigen
estimate of h-level l uses stream seed + 1 + l.
"""
import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from . import sip
from .basis import gauss, legendre_values
from .rng import uniform_pm1


# ------------------------------------------------------------ smoothers
def block_jacobi_blocks(A, nb):
    """Diagonal nb x nb blocks of A (element-block Jacobi, Sec. 6)."""
    n = A.shape[0] // nb
    out = np.empty((n, nb, nb))
    for e in range(n):
        s = slice(e * nb, (e + 1) * nb)
        out[e] = A[s, s].toarray()
    return out


def block_apply(inv_blocks, r):
    nb = inv_blocks.shape[1]
    return np.einsum("eij,ej->ei", inv_blocks, r.reshape(-1, nb)).ravel()


def invert_blocks(blocks):
    return np.linalg.inv(blocks)


def chebyshev(apply_A, apply_Minv, b, x0, steps, lmin, lmax):
    """Chebyshev iteration on M^{-1} A for the interval [lmin, lmax]
    (Saad Sec. 12.3 recurrence, preconditioned).  ``x0=None`` means a zero
    initial guess (no initial residual evaluation).  Returns the iterate
    after ``steps`` updates."""
    theta = 0.5 * (lmax + lmin)
    delta = 0.5 * (lmax - lmin)
    sigma = theta / delta
    if x0 is None:
        x = np.zeros_like(b)
        r = b.copy()
    else:
        x = x0.copy()
        r = b - apply_A(x)
    z = apply_Minv(r)
    rho = 1.0 / sigma
    d = z / theta
    for s in range(steps):
        x = x + d
        if s == steps - 1:
            break
        r = r - apply_A(d)
        z = apply_Minv(r)
        rho_new = 1.0 / (2.0 * sigma - rho)
        d = rho_new * rho * d + (2.0 * rho_new / delta) * z
        rho = rho_new
    return x


def estimate_lambda_max(apply_A, apply_Minv, n, seed, iters=10):
    """Largest Ritz value (real part) of ``iters`` Arnoldi steps of GMRES on
    M^{-1}A, started from M^{-1} b with b = SplitMix64 stream ``seed``."""
    b = uniform_pm1(seed, n)
    v = apply_Minv(b)
    m = min(iters, n)
    V = np.zeros((m + 1, n))
    H = np.zeros((m + 1, m))
    V[0] = v / np.linalg.norm(v)
    size = m
    for j in range(m):
        w = apply_Minv(apply_A(V[j]))
        for i in range(j + 1):                     # modified Gram-Schmidt
            H[i, j] = V[i] @ w
            w = w - H[i, j] * V[i]
        H[j + 1, j] = np.linalg.norm(w)
        if H[j + 1, j] <= 1e-14 * abs(H[j, j]):    # invariant subspace found
            size = j + 1
            break
        V[j + 1] = w / H[j + 1, j]
    ev = np.linalg.eigvals(H[:size, :size])
    return float(np.max(ev.real))


# ------------------------------------------------------------ transfers
def p_prolongation(k, ne, s=1):
    """P_k^s: coefficients of Q_s^2 (hierarchical modes i, j <= s) injected
    into Q_k^2, element by element; shape n_u(k) x n_u(s)."""
    n, m = k + 1, s + 1
    rows, cols = [], []
    for e in range(ne):
        for c in range(2):
            for j in range(m):
                for i in range(m):
                    rows.append(e * 2 * n * n + c * n * n + j * n + i)
                    cols.append(e * 2 * m * m + c * m * m + j * m + i)
    return sp.csr_matrix((np.ones(len(rows)), (rows, cols)), shape=(ne * 2 * n * n, ne * 2 * m * m))


def hat_1d(t, nodes_h, node):
    """Continuous piecewise-linear hat of ``node`` on a uniform grid."""
    return np.maximum(0.0, 1.0 - np.abs(t / nodes_h - node))


def continuous_to_dg(nx, ny, lx=1.0, ly=1.0):
    """P_cd: continuous bilinear (hat) coefficients at the (nx+1)(ny+1)
    vertices, dof 2*(vy*(nx+1)+vx)+c, -> discontinuous Q_1 modal
    coefficients (k = 1 numbering), by element-wise L2 projection of each
    hat function (exact for bilinears)."""
    hx, hy = lx / nx, ly / ny
    t, w = gauss(3)
    l1, _ = legendre_values(1, t)
    nv = (nx + 1) * (ny + 1)
    rows, cols, vals = [], [], []
    for ey in range(ny):
        for ex in range(nx):
            e = ey * nx + ex
            xq = ex * hx + (t + 1) * hx / 2
            yq = ey * hy + (t + 1) * hy / 2
            for vy in (ey, ey + 1):
                for vx in (ex, ex + 1):
                    hxv = hat_1d(xq, hx, vx)
                    hyv = hat_1d(yq, hy, vy)
                    # orthonormal reference basis: coefficient = int l_i l_j phi
                    cx = l1 @ (w * hxv)
                    cy = l1 @ (w * hyv)
                    for c in range(2):
                        for j in range(2):
                            for i in range(2):
                                rows.append(e * 8 + c * 4 + j * 2 + i)
                                cols.append(2 * (vy * (nx + 1) + vx) + c)
                                vals.append(cx[i] * cy[j])
    M = sp.coo_matrix((vals, (rows, cols)), shape=(nx * ny * 8, 2 * nv)).tocsr()
    M.sum_duplicates()
    M.eliminate_zeros()
    return M


def bilinear_prolongation(ncx, ncy):
    """P_h from the vertex grid of an ncx x ncy element mesh to that of the
    2ncx x 2ncy mesh: coarse hats evaluated at fine vertices; dof 2*v+c."""
    fx, fy = 2 * ncx, 2 * ncy
    rows, cols, vals = [], [], []
    for jy in range(fy + 1):
        for jx in range(fx + 1):
            for Iy in range(ncy + 1):
                wy = hat_1d(jy / 2.0, 1.0, Iy)
                if wy == 0.0:
                    continue
                for Ix in range(ncx + 1):
                    wx = hat_1d(jx / 2.0, 1.0, Ix)
                    if wx == 0.0:
                        continue
                    for c in range(2):
                        rows.append(2 * (jy * (fx + 1) + jx) + c)
                        cols.append(2 * (Iy * (ncx + 1) + Ix) + c)
                        vals.append(wx * wy)
    return sp.csr_matrix((vals, (rows, cols)), shape=(2 * (fx + 1) * (fy + 1), 2 * (ncx + 1) * (ncy + 1)))


# ------------------------------------------------------------ hierarchy
class HLevel:
    def __init__(self, A, P_to_finer, seed, steps):
        self.A = A.tocsr()
        self.P = P_to_finer              # prolongation from this level to the finer one
        self.dinv = 1.0 / self.A.diagonal()
        self.steps = steps
        self.lmax = estimate_lambda_max(lambda v: self.A @ v, lambda v: self.dinv * v,
                                        self.A.shape[0], seed)

    def smooth(self, b, x0):
        return chebyshev(lambda v: self.A @ v, lambda v: self.dinv * v, b, x0,
                         self.steps, 0.1 * self.lmax, 1.1 * self.lmax)


class HierarchyQ1:
    """Vertex-centred bilinear h-hierarchy: for A_1c on the mesh vertices
    (Sec. 6.1.2), or for A_0 on the element centres (Sec. 6.1.1); nx x ny
    intervals, 2 unknowns per vertex."""

    def __init__(self, A1c, nx, ny, n_coarsen, seed, steps=3):
        self.levels = []
        A = A1c.tocsr()
        cx, cy = nx, ny
        for l in range(n_coarsen):
            if cx % 2 or cy % 2:
                raise ValueError("mesh cannot be coarsened that many times")
            P = bilinear_prolongation(cx // 2, cy // 2)
            self.levels.append(HLevel(A, P, seed + 1 + l, steps))
            A = (P.T @ A @ P).tocsr()
            cx, cy = cx // 2, cy // 2
        self.coarse_A = A.toarray()
        self.coarse_lu = sla.lu_factor(self.coarse_A)

    def vcycle(self, b, l=0):
        if l == len(self.levels):
            return sla.lu_solve(self.coarse_lu, b)
        lev = self.levels[l]
        x = lev.smooth(b, None)
        r = b - lev.A @ x
        x = x + lev.P @ self.vcycle(lev.P.T @ r, l + 1)
        return lev.smooth(b, x)


class HPMultigrid:
    """Algorithm 1 with the p-coarse space Q^2_1 or Q^2_0 (one cycle, y0 = 0).

    coarse = "q1": n_hlevels = 0: coarse problem A_1 solved by LU
    (A_p(Q^2_1)); n_hlevels > 0: coarse correction P_cd V_h(R_dc r)
    (A_hp(Q^2_1)).
    coarse = "q0" (Sec. 6.1.1): the coarse space is the element-wise
    constants, A_0 = P^T A P (a 5-point stencil per component); with
    n_hlevels > 0 it is coarsened as a vertex grid of the element centres
    (an odd number of elements per side), bilinear R_h = P_h^T, Galerkin
    coarse operators, Chebyshev / point-Jacobi smoothing, LU at the
    coarsest level (A_hp(Q^2_0)); n_hlevels = 0: LU of A_0 (A_p(Q^2_0))."""

    def __init__(self, prob, A, n_hlevels, seed, p_steps=2, h_steps=3, blocks=None,
                 coarse="q1"):
        k, nb = prob.k, prob.num.nb
        self.A = A.tocsr()
        self.steps = p_steps
        if blocks is None:
            blocks = block_jacobi_blocks(self.A, nb)
        self.inv_blocks = invert_blocks(blocks)
        self.Minv = lambda r: block_apply(self.inv_blocks, r)
        self.lmax = estimate_lambda_max(lambda v: self.A @ v, self.Minv, self.A.shape[0], seed)
        self.coarse = coarse
        self.n_hlevels = n_hlevels
        if coarse == "q0":
            self.P = p_prolongation(k, prob.num.ne, 0)
            self.A0 = (self.P.T @ self.A @ self.P).tocsr()
            if n_hlevels == 0:
                self.coarse_lu = sla.lu_factor(self.A0.toarray())
            else:
                # element centres as the vertices of an (nx-1) x (ny-1) grid
                self.h = HierarchyQ1(self.A0, prob.nx - 1, prob.ny - 1, n_hlevels, seed, h_steps)
            return
        self.P = p_prolongation(k, prob.num.ne, 1)
        self.A1 = (self.P.T @ self.A @ self.P).tocsr()
        if n_hlevels == 0:
            self.coarse_lu = sla.lu_factor(self.A1.toarray())
        else:
            self.Pcd = continuous_to_dg(prob.nx, prob.ny, prob.lx, prob.ly)
            self.A1c = (self.Pcd.T @ self.A1 @ self.Pcd).tocsr()
            self.h = HierarchyQ1(self.A1c, prob.nx, prob.ny, n_hlevels, seed, h_steps)

    def smooth(self, b, x0):
        return chebyshev(lambda v: self.A @ v, self.Minv, b, x0, self.steps,
                         0.1 * self.lmax, 1.1 * self.lmax)

    def coarse_solve(self, rc):
        if self.n_hlevels == 0:
            return sla.lu_solve(self.coarse_lu, rc)
        if self.coarse == "q0":
            return self.h.vcycle(rc)
        return self.Pcd @ self.h.vcycle(self.Pcd.T @ rc)

    def __call__(self, b):
        y = self.smooth(b, None)
        r = b - self.A @ y
        y = y + self.P @ self.coarse_solve(self.P.T @ r)
        return self.smooth(b, y)
