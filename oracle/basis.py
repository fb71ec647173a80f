"""Orthonormal hierarchical Legendre basis and Gauss quadrature (oracle).

Test infrastructure only (see ``oracle/__init__``).

Sec. 5 ("tensor products of pairwise orthogonal Legendre polynomials") and
the remark that S* is diagonal because the basis is orthonormal fix the
basis up to normalisation; we take l_i = sqrt((2i+1)/2) P_i on [-1, 1], so
that the basis is orthonormal on the reference square.  A velocity basis
function on element K is phi_{c,j,i}(x, y) = l_i(xi(x)) l_j(zeta(y)) e_c,
pressure psi_{j,i} = l_i(xi) l_j(zeta) with i, j < k.

Values are produced by ``numpy.polynomial.legendre`` (a library primitive),
never by closed-form tables, so the oracle shares no formula with the
CUDA tables.
"""
import numpy as np
from numpy.polynomial import legendre as npleg


def gauss(npts):
    """Gauss-Legendre points and weights on [-1, 1] (library primitive)."""
    return npleg.leggauss(npts)


def legendre_values(order, xi):
    """Orthonormal l_0..l_order and their d/dxi at reference points ``xi``.

    Returns (val, der) with shape (order+1, len(xi)).
    """
    xi = np.asarray(xi, dtype=np.float64)
    val = np.empty((order + 1, xi.size))
    der = np.empty((order + 1, xi.size))
    for i in range(order + 1):
        coef = np.zeros(i + 1)
        coef[i] = 1.0
        scale = np.sqrt((2.0 * i + 1.0) / 2.0)
        val[i] = scale * npleg.legval(xi, coef)
        der[i] = scale * npleg.legval(xi, npleg.legder(coef)) if i > 0 else 0.0
    return val, der


class Numbering:
    """Global dof numbering for the DG spaces of Sec. 4.

    Velocity: element e = ey*nx + ex owns a contiguous block of
    2 (k+1)^2 dofs ordered [c][j][i] (c = component, i = x-degree fastest).
    Pressure: element e owns k^2 dofs ordered [j][i].
    """

    def __init__(self, nx, ny, k):
        self.nx, self.ny, self.k = nx, ny, k
        self.n = k + 1
        self.nb = 2 * self.n * self.n
        self.mp = k * k
        self.ne = nx * ny
        self.n_u = self.ne * self.nb
        self.n_p = self.ne * self.mp

    def elem(self, ex, ey):
        return ey * self.nx + ex

    def u_dofs(self, e):
        return np.arange(e * self.nb, (e + 1) * self.nb)

    def p_dofs(self, e):
        return np.arange(e * self.mp, (e + 1) * self.mp)


class ElementGeometry:
    """Affine map of element (ex, ey) of an nx x ny grid on [0,lx]x[0,ly]."""

    def __init__(self, nx, ny, lx, ly):
        self.nx, self.ny, self.lx, self.ly = nx, ny, lx, ly
        self.hx = lx / nx
        self.hy = ly / ny

    def origin(self, ex, ey):
        return ex * self.hx, ey * self.hy

    def to_ref(self, ex, ey, x, y):
        x0, y0 = self.origin(ex, ey)
        return 2.0 * (x - x0) / self.hx - 1.0, 2.0 * (y - y0) / self.hy - 1.0


def velocity_basis_at(k, geom, ex, ey, x, y):
    """Velocity basis of element (ex, ey) at physical points (x, y).

    Returns (U, GU): U[f, q, c] is component c of basis function f at point
    q; GU[f, q, c, d] = d u_c / d x_d.  Function index f = c*n*n + j*n + i.
    """
    n = k + 1
    xi, zeta = geom.to_ref(ex, ey, np.asarray(x), np.asarray(y))
    lx, dlx = legendre_values(k, xi)
    ly, dly = legendre_values(k, zeta)
    dlx = dlx * (2.0 / geom.hx)
    dly = dly * (2.0 / geom.hy)
    nq = xi.size
    U = np.zeros((2 * n * n, nq, 2))
    GU = np.zeros((2 * n * n, nq, 2, 2))
    for c in range(2):
        for j in range(n):
            for i in range(n):
                f = c * n * n + j * n + i
                U[f, :, c] = lx[i] * ly[j]
                GU[f, :, c, 0] = dlx[i] * ly[j]
                GU[f, :, c, 1] = lx[i] * dly[j]
    return U, GU


def pressure_basis_at(k, geom, ex, ey, x, y):
    """Pressure basis (degree k-1 per variable) at physical points."""
    xi, zeta = geom.to_ref(ex, ey, np.asarray(x), np.asarray(y))
    if k < 1:
        raise ValueError("k must be >= 1")
    lx, _ = legendre_values(k - 1, xi)
    ly, _ = legendre_values(k - 1, zeta)
    P = np.zeros((k * k, xi.size))
    for j in range(k):
        for i in range(k):
            P[j * k + i] = lx[i] * ly[j]
    return P
