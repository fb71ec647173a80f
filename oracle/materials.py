"""Element-wise material rasterisation (oracle side).

Test infrastructure only (see ``oracle/__init__``).

Sec. 7.3 (sedimenting inclusions): a Cartesian grid cannot resolve the
inclusions, so each element takes the maximum viscosity and the minimum
density found inside it.  Elements are open sets (Sec. 3); an inclusion is
closed.  With eta(x) = max(eta_bg, eta_i over the inclusions containing x):
  eta_K = max over the open cell,   rho_K = min over the open cell.
Reading used for rho: an element takes an inclusion's density only when the
whole cell lies inside that single inclusion (overlaps of several discs
covering a cell are not merged).

Written independently of the CUDA rasteriser: the oracle tests the geometry
by brute force on point clouds in the pins; here it uses the closed-form
distance from a disc centre to the closed cell.
"""
import numpy as np


def _cells(nx, ny, lx, ly):
    hx, hy = lx / nx, ly / ny
    ex, ey = np.meshgrid(np.arange(nx), np.arange(ny), indexing="xy")
    x0 = ex.ravel() * hx
    y0 = ey.ravel() * hy
    return x0, y0, x0 + hx, y0 + hy


def rasterise_discs(nx, ny, discs, eta_bg=1.0, rho_bg=1.0, lx=1.0, ly=1.0):
    """discs: iterable of (cx, cy, r, eta_i, rho_i) with eta_i >= eta_bg and
    rho_i >= rho_bg (heavy, stiff inclusions as in Sec. 7.3).  Returns
    (eta, rho), each of length nx*ny in element order e = ey*nx + ex."""
    x0, y0, x1, y1 = _cells(nx, ny, lx, ly)
    for d in discs:
        if d[3] < eta_bg or d[4] < rho_bg:
            raise ValueError("inclusions must be at least as viscous and dense as the background")
    eta = np.full(x0.size, float(eta_bg))
    rho = np.full(x0.size, float(rho_bg))
    for cx, cy, r, eta_i, rho_i in discs:
        dx = np.maximum(np.maximum(x0 - cx, cx - x1), 0.0)
        dy = np.maximum(np.maximum(y0 - cy, cy - y1), 0.0)
        meets = dx * dx + dy * dy < r * r              # open cell meets closed disc
        eta = np.where(meets, np.maximum(eta, eta_i), eta)
        fx = np.maximum(np.abs(x0 - cx), np.abs(x1 - cx))
        fy = np.maximum(np.abs(y0 - cy), np.abs(y1 - cy))
        inside = fx * fx + fy * fy <= r * r            # farthest corner inside
        rho = np.where(inside, np.maximum(rho, rho_i), rho)
    return eta, rho


def rasterise_box(nx, ny, box, eta_in, rho_in, eta_bg=1.0, rho_bg=1.0, lx=1.0, ly=1.0):
    """A closed axis-aligned box inclusion box = (xa, xb, ya, yb)."""
    xa, xb, ya, yb = box
    x0, y0, x1, y1 = _cells(nx, ny, lx, ly)
    meets = (x0 < xb) & (x1 > xa) & (y0 < yb) & (y1 > ya)
    inside = (x0 >= xa) & (x1 <= xb) & (y0 >= ya) & (y1 <= yb)
    eta = np.where(meets, max(eta_in, eta_bg), eta_bg).astype(np.float64)
    rho = np.where(inside, rho_in, rho_bg).astype(np.float64)
    return eta, rho


def rasterise_inclusions(nx, ny, shapes, eta_bg=1.0, rho_bg=1.0, lx=1.0, ly=1.0):
    """Records (kind, a, b, c, d, eta_i, rho_i): kind 0 = disc centre (a, b)
    radius c; kind 1 = box [a, b] x [c, d].  Combines the per-shape results
    by element-wise max (both eta and rho grow with every inclusion)."""
    eta = np.full(nx * ny, float(eta_bg))
    rho = np.full(nx * ny, float(rho_bg))
    for kind, a, b, c, d, e_i, r_i in np.asarray(shapes, dtype=np.float64).reshape(-1, 7):
        if kind == 0:
            e1, r1 = rasterise_discs(nx, ny, [(a, b, c, e_i, r_i)], eta_bg, rho_bg, lx, ly)
        else:
            e1, r1 = rasterise_box(nx, ny, (a, b, c, d), e_i, r_i, eta_bg, rho_bg, lx, ly)
        eta = np.maximum(eta, e1)
        rho = np.maximum(rho, r1)
    return eta, rho
