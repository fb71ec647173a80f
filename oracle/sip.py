"""Explicit FP64 assembly of the SIP-DG Stokes operators (oracle).

Test infrastructure only (see ``oracle/__init__``).

Everything here is the paper's weak form written out and integrated by
Gauss-Legendre quadrature at physical points:

* ``assemble_A``   eq. stiffness_form (Sec. 4): volume 2 eta eps(u):eps(v),
  interior-face consistency / symmetry / penalty terms, Navier-face terms.
* ``assemble_B``   eq. divergence_form (Sec. 4).
* ``rhs_force``    eq. rhs_f (Sec. 4), f(v) = sum_K int_K f . v.
* ``schur_mass``   S* of Sec. 5: the pressure mass matrix scaled by 1/eta_K.
* ``penalty``      sigma_e = gamma_e C_e with gamma_e = n_f eta_e (1+tau) x
  {1 interior, 2 Navier}, n_f = 4, tau = 0 (Lemma 4.4 eq. sipg_penalty and
  the remark that tau is zero in the computations); C_e from the discrete
  trace inequality C_K = (k+1)^2 |e|/|K| (Lemma 4.1) maximised over the two
  neighbours (eq. const_trace_face); eta_e from eq. eta_face.

Boundary conditions per side (left, right, bottom, top):
  'navier'    u.n = 0, t.2 eta eps(u) n = 0, weakly (the paper's Navier terms)
  'neumann'   natural, no face terms
  'dirichlet' homogeneous u = 0 imposed by the symmetric Nitsche analogue of
              the interior terms with a zero exterior trace (not in the paper:
              -int (2 eta eps(u) n).v - int (2 eta eps(v) n).u + sigma int u.v
              with the Navier factor 2 in sigma, and int q (u.n) in b_h).
"""
from dataclasses import dataclass, field

import numpy as np
import scipy.sparse as sp

from .basis import (Numbering, ElementGeometry, gauss, velocity_basis_at,
                    pressure_basis_at)

SIDES = ("left", "right", "bottom", "top")
N_FACES = 4          # n_f in eq. sipg_penalty (faces of a quadrilateral)
TAU = 0.0            # tau in eq. sipg_penalty ("set to zero")


@dataclass
class Problem:
    """A Stokes problem on an nx x ny Cartesian grid of [0,lx]x[0,ly].

    ``eta`` is element-wise constant (assumption ASh1), indexed e = ey*nx+ex.
    ``k_penalty`` is the degree used in the trace constant (defaults to k);
    the Galerkin coarse operator A_1 keeps the fine degree there.
    """
    nx: int
    ny: int
    k: int
    eta: np.ndarray
    bc: tuple = ("navier", "navier", "navier", "navier")
    lx: float = 1.0
    ly: float = 1.0
    penalty_scale: float = 1.0
    k_penalty: int = None
    num: Numbering = field(init=False, repr=False)
    geom: ElementGeometry = field(init=False, repr=False)

    def __post_init__(self):
        self.eta = np.asarray(self.eta, dtype=np.float64).reshape(-1)
        if self.eta.size != self.nx * self.ny:
            raise ValueError("eta must have nx*ny entries")
        if self.k_penalty is None:
            self.k_penalty = self.k
        self.num = Numbering(self.nx, self.ny, self.k)
        self.geom = ElementGeometry(self.nx, self.ny, self.lx, self.ly)

    @property
    def has_neumann(self):
        return "neumann" in self.bc


# ---------------------------------------------------------------- penalty
def trace_constant(prob, face_len):
    """C_K = (k+1)^2 |e| / |K| (Lemma 4.1, eq. discrete_trace_constant)."""
    area = prob.geom.hx * prob.geom.hy
    return (prob.k_penalty + 1) ** 2 * face_len / area


def penalty(prob, eta_minus, eta_plus=None, face_len=1.0):
    """sigma_e = gamma_e C_e, eq. sipg_penalty taken at its lower bound.

    Interior face: eta_e = max(eta+, eta-) (eq. eta_face), factor 1;
    boundary (Navier, and the Dirichlet extension): eta_e = eta_K, factor 2.
    All elements have the same shape, so C_e = max(C_K+, C_K-) = C_K.
    """
    c_e = trace_constant(prob, face_len)
    if eta_plus is None:
        eta_e, factor = eta_minus, 2.0
    else:
        eta_e, factor = max(eta_minus, eta_plus), 1.0
    gamma = N_FACES * eta_e * (1.0 + TAU) * factor
    return prob.penalty_scale * gamma * c_e


# ------------------------------------------------------------- geometry
def _face_points(prob, ex, ey, side, npts):
    """Physical quadrature points / weights on a side of element (ex, ey)
    and the outward unit normal of that element there."""
    g = prob.geom
    x0, y0 = g.origin(ex, ey)
    t, w = gauss(npts)
    if side in ("left", "right"):
        x = np.full(npts, x0 if side == "left" else x0 + g.hx)
        y = y0 + (t + 1.0) * g.hy / 2.0
        wq = w * g.hy / 2.0
        nrm = np.array([-1.0, 0.0]) if side == "left" else np.array([1.0, 0.0])
        length = g.hy
    else:
        y = np.full(npts, y0 if side == "bottom" else y0 + g.hy)
        x = x0 + (t + 1.0) * g.hx / 2.0
        wq = w * g.hx / 2.0
        nrm = np.array([0.0, -1.0]) if side == "bottom" else np.array([0.0, 1.0])
        length = g.hx
    return x, y, wq, nrm, length


def _volume_points(prob, ex, ey, npts):
    g = prob.geom
    x0, y0 = g.origin(ex, ey)
    t, w = gauss(npts)
    X, Y = np.meshgrid(x0 + (t + 1) * g.hx / 2, y0 + (t + 1) * g.hy / 2,
                       indexing="ij")
    W = np.outer(w, w) * (g.hx * g.hy / 4.0)
    return X.ravel(), Y.ravel(), W.ravel()


def _strain(GU):
    return 0.5 * (GU + np.swapaxes(GU, -1, -2))


def neighbour(prob, ex, ey, side):
    """Element across ``side`` of (ex, ey), or None at the boundary."""
    dx, dy = {"left": (-1, 0), "right": (1, 0), "bottom": (0, -1), "top": (0, 1)}[side]
    fx, fy = ex + dx, ey + dy
    if 0 <= fx < prob.nx and 0 <= fy < prob.ny:
        return fx, fy
    return None


def boundary_type(prob, side):
    return prob.bc[SIDES.index(side)]


# ------------------------------------------------------------- A blocks
def volume_block_A(prob, ex, ey):
    """int_K 2 eta eps(u_h) : eps(v_h) dx for all basis pairs of K."""
    q = prob.k + 2
    X, Y, W = _volume_points(prob, ex, ey, q)
    _, GU = velocity_basis_at(prob.k, prob.geom, ex, ey, X, Y)
    E = _strain(GU)
    eta = prob.eta[prob.num.elem(ex, ey)]
    return np.einsum("fqcd,gqcd,q->fg", E, E, 2.0 * eta * W)


def interior_face_A(prob, ex, ey, side):
    """Interior-face part of eq. stiffness_form on the face between K- =
    (ex, ey) and K+ across ``side``.

    Returns the (2 nb) x (2 nb) matrix over [basis of K-, basis of K+]
    (rows = test v_h, columns = trial u_h) of
      - {2 eta eps(u)} : [[v (x) n]] - {2 eta eps(v)} : [[u (x) n]]
      + sigma_e [[u (x) n]] : [[v (x) n]].
    """
    nb_ = neighbour(prob, ex, ey, side)
    fx, fy = nb_
    q = prob.k + 2
    x, y, wq, nrm, length = _face_points(prob, ex, ey, side, q)
    em, ep = prob.num.elem(ex, ey), prob.num.elem(fx, fy)
    Um, GUm = velocity_basis_at(prob.k, prob.geom, ex, ey, x, y)
    Up, GUp = velocity_basis_at(prob.k, prob.geom, fx, fy, x, y)
    U = np.concatenate([Um, Up])
    # each basis function lives on one side: its jump is u_side (x) n_side
    # and its average is half of its own 2 eta eps(u).
    S = np.concatenate([2.0 * prob.eta[em] * _strain(GUm),
                        2.0 * prob.eta[ep] * _strain(GUp)])
    nside = np.concatenate([np.tile(nrm, (Um.shape[0], 1)),
                            np.tile(-nrm, (Up.shape[0], 1))])
    J = np.einsum("fqc,fd->fqcd", U, nside)
    Avg = 0.5 * S
    sigma = penalty(prob, prob.eta[em], prob.eta[ep], length)
    cons = np.einsum("gqcd,fqcd,q->fg", Avg, J, wq)      # {2 eta eps(u)} : [[v n]]
    pen = np.einsum("gqcd,fqcd,q->fg", J, J, wq)
    return -cons - cons.T + sigma * pen


def boundary_face_A(prob, ex, ey, side):
    """Boundary-face part of eq. stiffness_form for the face ``side`` of K."""
    kind = boundary_type(prob, side)
    nb = prob.num.nb
    if kind == "neumann":
        return np.zeros((nb, nb))
    q = prob.k + 2
    x, y, wq, nrm, length = _face_points(prob, ex, ey, side, q)
    e = prob.num.elem(ex, ey)
    U, GU = velocity_basis_at(prob.k, prob.geom, ex, ey, x, y)
    S = 2.0 * prob.eta[e] * _strain(GU)
    sigma = penalty(prob, prob.eta[e], None, length)
    Sn = np.einsum("fqcd,d->fqc", S, nrm)               # 2 eta eps(u) n
    if kind == "navier":
        nSn = np.einsum("fqc,c->fq", Sn, nrm)           # n . 2 eta eps(u) n
        un = np.einsum("fqc,c->fq", U, nrm)             # u . n
        cons = np.einsum("gq,fq,q->fg", nSn, un, wq)
        pen = np.einsum("gq,fq,q->fg", un, un, wq)
    elif kind == "dirichlet":
        cons = np.einsum("gqc,fqc,q->fg", Sn, U, wq)
        pen = np.einsum("gqc,fqc,q->fg", U, U, wq)
    else:
        raise ValueError(kind)
    return -cons - cons.T + sigma * pen


def _faces(prob):
    """Yield ('interior', ex, ey, side) for right/top interior faces and
    ('boundary', ex, ey, side) for every boundary face."""
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            for side in SIDES:
                if neighbour(prob, ex, ey, side) is None:
                    yield "boundary", ex, ey, side
                elif side in ("right", "top"):
                    yield "interior", ex, ey, side


def assemble_A(prob):
    """The SIP viscous matrix A (eq. stiffness_form), CSR, FP64."""
    num = prob.num
    rows, cols, vals = [], [], []

    def add(rdofs, cdofs, blk):
        r, c = np.meshgrid(rdofs, cdofs, indexing="ij")
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(blk.ravel())

    for ey in range(prob.ny):
        for ex in range(prob.nx):
            d = num.u_dofs(num.elem(ex, ey))
            add(d, d, volume_block_A(prob, ex, ey))
    for kind, ex, ey, side in _faces(prob):
        e = num.elem(ex, ey)
        if kind == "boundary":
            d = num.u_dofs(e)
            add(d, d, boundary_face_A(prob, ex, ey, side))
        else:
            fx, fy = neighbour(prob, ex, ey, side)
            d = np.concatenate([num.u_dofs(e), num.u_dofs(num.elem(fx, fy))])
            add(d, d, interior_face_A(prob, ex, ey, side))
    A = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(num.n_u, num.n_u)).tocsr()
    A.sum_duplicates()
    return A


def element_rows_A(prob, ex, ey):
    """The rows of A belonging to element (ex, ey), built on their own.

    Returns {element index: nb x nb block} for the element and its face
    neighbours; used to check single outputs of a large apply one by one.
    """
    num = prob.num
    e = num.elem(ex, ey)
    nb = num.nb
    blocks = {e: volume_block_A(prob, ex, ey)}
    for side in SIDES:
        nbr = neighbour(prob, ex, ey, side)
        if nbr is None:
            blocks[e] = blocks[e] + boundary_face_A(prob, ex, ey, side)
        else:
            F = interior_face_A(prob, ex, ey, side)
            f = num.elem(*nbr)
            blocks[e] = blocks[e] + F[:nb, :nb]
            blocks[f] = blocks.get(f, 0) + F[:nb, nb:]
    return blocks


# ------------------------------------------------------------- B blocks
def assemble_B(prob):
    """B with B[v, q] = b_h(v, q) (eq. divergence_form); shape n_u x n_p."""
    num, k = prob.num, prob.k
    rows, cols, vals = [], [], []

    def add(rdofs, cdofs, blk):
        r, c = np.meshgrid(rdofs, cdofs, indexing="ij")
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(blk.ravel())

    for ey in range(prob.ny):
        for ex in range(prob.nx):
            e = num.elem(ex, ey)
            add(num.u_dofs(e), num.p_dofs(e), volume_block_B(prob, ex, ey))
    for kind, ex, ey, side in _faces(prob):
        e = num.elem(ex, ey)
        if kind == "boundary":
            add(num.u_dofs(e), num.p_dofs(e), boundary_face_B(prob, ex, ey, side))
        else:
            fx, fy = neighbour(prob, ex, ey, side)
            f = num.elem(fx, fy)
            du = np.concatenate([num.u_dofs(e), num.u_dofs(f)])
            dp = np.concatenate([num.p_dofs(e), num.p_dofs(f)])
            add(du, dp, interior_face_B(prob, ex, ey, side))
    B = sp.coo_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))),
                      shape=(num.n_u, num.n_p)).tocsr()
    B.sum_duplicates()
    return B


def volume_block_B(prob, ex, ey):
    """int_K -div(v) q dx."""
    X, Y, W = _volume_points(prob, ex, ey, prob.k + 2)
    _, GU = velocity_basis_at(prob.k, prob.geom, ex, ey, X, Y)
    P = pressure_basis_at(prob.k, prob.geom, ex, ey, X, Y)
    div = GU[:, :, 0, 0] + GU[:, :, 1, 1]
    return -np.einsum("fq,gq,q->fg", div, P, W)


def interior_face_B(prob, ex, ey, side):
    """int_e {q} [[v . n]] over [K-, K+] x [K-, K+]."""
    fx, fy = neighbour(prob, ex, ey, side)
    x, y, wq, nrm, _ = _face_points(prob, ex, ey, side, prob.k + 2)
    Um, _ = velocity_basis_at(prob.k, prob.geom, ex, ey, x, y)
    Up, _ = velocity_basis_at(prob.k, prob.geom, fx, fy, x, y)
    Pm = pressure_basis_at(prob.k, prob.geom, ex, ey, x, y)
    Pp = pressure_basis_at(prob.k, prob.geom, fx, fy, x, y)
    jump = np.concatenate([np.einsum("fqc,c->fq", Um, nrm),
                           np.einsum("fqc,c->fq", Up, -nrm)])
    avg = 0.5 * np.concatenate([Pm, Pp])
    return np.einsum("fq,gq,q->fg", jump, avg, wq)


def boundary_face_B(prob, ex, ey, side):
    """int_e q (v . n) on Navier (and Dirichlet) faces; 0 on Neumann."""
    kind = boundary_type(prob, side)
    if kind == "neumann":
        return np.zeros((prob.num.nb, prob.num.mp))
    x, y, wq, nrm, _ = _face_points(prob, ex, ey, side, prob.k + 2)
    U, _ = velocity_basis_at(prob.k, prob.geom, ex, ey, x, y)
    P = pressure_basis_at(prob.k, prob.geom, ex, ey, x, y)
    un = np.einsum("fqc,c->fq", U, nrm)
    return np.einsum("fq,gq,q->fg", un, P, wq)


def element_rows_B(prob, ex, ey):
    """Rows of B for the velocity dofs of (ex, ey): {element: nb x mp}."""
    num = prob.num
    e = num.elem(ex, ey)
    nb, mp = num.nb, num.mp
    blocks = {e: volume_block_B(prob, ex, ey)}
    for side in SIDES:
        nbr = neighbour(prob, ex, ey, side)
        if nbr is None:
            blocks[e] = blocks[e] + boundary_face_B(prob, ex, ey, side)
        else:
            F = interior_face_B(prob, ex, ey, side)
            f = num.elem(*nbr)
            blocks[e] = blocks[e] + F[:nb, :mp]
            blocks[f] = blocks.get(f, 0) + F[:nb, mp:]
    return blocks


def element_cols_B(prob, ex, ey):
    """Rows of B^T for the pressure dofs of (ex, ey): {element: mp x nb}."""
    num = prob.num
    e = num.elem(ex, ey)
    nb, mp = num.nb, num.mp
    blocks = {e: volume_block_B(prob, ex, ey).T}
    for side in SIDES:
        nbr = neighbour(prob, ex, ey, side)
        if nbr is None:
            blocks[e] = blocks[e] + boundary_face_B(prob, ex, ey, side).T
        else:
            F = interior_face_B(prob, ex, ey, side)
            f = num.elem(*nbr)
            blocks[e] = blocks[e] + F[:nb, :mp].T
            blocks[f] = blocks.get(f, 0) + F[nb:, :mp].T
    return blocks


# ------------------------------------------------------------ rhs, S*
def rhs_force(prob, force, npts=None):
    """f(v) = sum_K int_K f . v (eq. rhs_f) for a callable force(x, y) ->
    (fx, fy), by (k+4)-point Gauss quadrature per direction."""
    num = prob.num
    q = npts or prob.k + 4
    f = np.zeros(num.n_u)
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            X, Y, W = _volume_points(prob, ex, ey, q)
            U, _ = velocity_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            fx, fy = force(X, Y)
            F = np.stack([np.broadcast_to(fx, X.shape), np.broadcast_to(fy, X.shape)], -1)
            f[num.u_dofs(num.elem(ex, ey))] = np.einsum("fqc,qc,q->f", U, F, W)
    return f


def rhs_body_force(prob, rho, g=10.0):
    """f = (0, -g rho_K), element-wise constant density (Sec. 7.3)."""
    rho = np.asarray(rho, dtype=np.float64).reshape(-1)

    num = prob.num
    f = np.zeros(num.n_u)
    q = prob.k + 2
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            e = num.elem(ex, ey)
            X, Y, W = _volume_points(prob, ex, ey, q)
            U, _ = velocity_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            f[num.u_dofs(e)] = np.einsum("fq,q->f", U[:, :, 1], W) * (-g * rho[e])
    return f


def pressure_mass(prob):
    """int psi_a psi_b per element, diagonal entries (the basis is
    orthonormal on the reference square, so the matrix is diagonal; the
    assembled off-diagonal part is checked by a pin)."""
    num = prob.num
    out = np.zeros(num.n_p)
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            X, Y, W = _volume_points(prob, ex, ey, prob.k + 2)
            P = pressure_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            out[num.p_dofs(num.elem(ex, ey))] = np.einsum("fq,fq,q->f", P, P, W)
    return out


def pressure_mass_block(prob, ex, ey):
    """Full element pressure mass block (used by the diagonality pin)."""
    X, Y, W = _volume_points(prob, ex, ey, prob.k + 2)
    P = pressure_basis_at(prob.k, prob.geom, ex, ey, X, Y)
    return np.einsum("fq,gq,q->fg", P, P, W)


def schur_mass(prob):
    """Diagonal of S* = pressure mass scaled by 1/eta_K (Sec. 5)."""
    m = pressure_mass(prob)
    eta_p = np.repeat(prob.eta, prob.num.mp)
    return m / eta_p


def pressure_constant(prob):
    """Coefficients of the constant pressure 1 (the null vector of B when
    there is no Neumann face), by L2 projection."""
    num = prob.num
    out = np.zeros(num.n_p)
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            X, Y, W = _volume_points(prob, ex, ey, prob.k + 2)
            P = pressure_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            M = np.einsum("fq,gq,q->fg", P, P, W)
            out[num.p_dofs(num.elem(ex, ey))] = np.linalg.solve(M, P @ W)
    return out


def project_velocity(prob, func, npts=None):
    """L2 projection of a velocity field func(x,y)->(ux,uy) onto V_h."""
    num = prob.num
    q = npts or prob.k + 4
    out = np.zeros(num.n_u)
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            X, Y, W = _volume_points(prob, ex, ey, q)
            U, _ = velocity_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            ux, uy = func(X, Y)
            F = np.stack([np.broadcast_to(ux, X.shape), np.broadcast_to(uy, X.shape)], -1)
            M = np.einsum("fqc,gqc,q->fg", U, U, W)
            out[num.u_dofs(num.elem(ex, ey))] = np.linalg.solve(M, np.einsum("fqc,qc,q->f", U, F, W))
    return out


def project_pressure(prob, func, npts=None):
    """L2 projection of a scalar func(x,y) onto Q_h."""
    num = prob.num
    q = npts or prob.k + 4
    out = np.zeros(num.n_p)
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            X, Y, W = _volume_points(prob, ex, ey, q)
            P = pressure_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            M = np.einsum("fq,gq,q->fg", P, P, W)
            out[num.p_dofs(num.elem(ex, ey))] = np.linalg.solve(M, P @ (func(X, Y) * W))
    return out


def l2_errors(prob, u, p, u_exact, p_exact, npts=None):
    """||u - u_h||_L2 and ||p - p_h||_L2 by (k+4)-point quadrature."""
    num = prob.num
    q = npts or prob.k + 4
    eu = ep = 0.0
    for ey in range(prob.ny):
        for ex in range(prob.nx):
            e = num.elem(ex, ey)
            X, Y, W = _volume_points(prob, ex, ey, q)
            U, _ = velocity_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            P = pressure_basis_at(prob.k, prob.geom, ex, ey, X, Y)
            uh = np.einsum("fqc,f->qc", U, u[num.u_dofs(e)])
            ph = P.T @ p[num.p_dofs(e)]
            ux, uy = u_exact(X, Y)
            eu += np.sum(W * ((ux - uh[:, 0]) ** 2 + (uy - uh[:, 1]) ** 2))
            ep += np.sum(W * (p_exact(X, Y) - ph) ** 2)
    return np.sqrt(eu), np.sqrt(ep)
