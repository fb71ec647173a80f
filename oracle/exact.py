"""Manufactured solutions for the convergence-rate and patch pins (oracle).

Test infrastructure only (see ``oracle/__init__``).

The paper's SolCx closed form is only cited, not printed, so its place is
taken by solutions built here from stream functions (velocity = curl psi is
divergence free) with the force f = -div(2 eta eps(u)) + grad p of
eq. momentum_balance.  Each is checked against finite differences in the pins.
"""
import numpy as np
from numpy.polynomial import Polynomial

PI = np.pi


class SmoothNavier:
    """psi = sin(pi x) sin(pi y) on the unit square, constant eta,
    p = cos(pi x) cos(pi y).  u.n = 0 and eps_xy = 0 on every side, so the
    homogeneous Navier conditions hold; p has zero mean."""

    def __init__(self, eta=1.0):
        self.eta = eta

    def u(self, x, y):
        return (PI * np.sin(PI * x) * np.cos(PI * y),
                -PI * np.cos(PI * x) * np.sin(PI * y))

    def p(self, x, y):
        return np.cos(PI * x) * np.cos(PI * y)

    def f(self, x, y):
        ux, uy = self.u(x, y)
        # -eta lap u = 2 pi^2 eta u for this psi
        return (2 * PI ** 2 * self.eta * ux - PI * np.sin(PI * x) * np.cos(PI * y),
                2 * PI ** 2 * self.eta * uy - PI * np.cos(PI * x) * np.sin(PI * y))


class JumpNavier(SmoothNavier):
    """Viscosity eta1 for x < xc, eta2 for x > xc (Navier on all sides).

    Same velocity; p = 2 eta(x) du_x/dx + cos(pi x) cos(pi y).  Then
    sigma_xx = -cos cos and sigma_xy = 0 are continuous across x = xc, so u, p
    solve the weak problem with the side-wise force -eta lap u + grad p."""

    def __init__(self, eta1, eta2, xc=0.25):
        self.eta1, self.eta2, self.xc = eta1, eta2, xc

    def etax(self, x):
        return np.where(x < self.xc, self.eta1, self.eta2)

    def p(self, x, y):
        dux = PI ** 2 * np.cos(PI * x) * np.cos(PI * y)
        return 2 * self.etax(x) * dux + np.cos(PI * x) * np.cos(PI * y)

    def f(self, x, y):
        ux, uy = self.u(x, y)
        eta = self.etax(x)
        c = 2 * eta * PI ** 2
        dpx = -2 * eta * PI ** 3 * np.sin(PI * x) * np.cos(PI * y) - PI * np.sin(PI * x) * np.cos(PI * y)
        dpy = -2 * eta * PI ** 3 * np.cos(PI * x) * np.sin(PI * y) - PI * np.cos(PI * x) * np.sin(PI * y)
        return c * ux + dpx, c * uy + dpy

    def eta_elements(self, nx, ny):
        hx = 1.0 / nx
        xc = (np.arange(nx) + 0.5) * hx
        return np.tile(self.etax(xc), ny)


class SmoothDirichlet:
    """psi = sin^2(pi x) sin^2(pi y): u = 0 on the boundary, constant eta,
    p = cos(pi x) cos(pi y) (zero mean)."""

    def __init__(self, eta=1.0):
        self.eta = eta

    def u(self, x, y):
        return (PI * np.sin(PI * x) ** 2 * np.sin(2 * PI * y),
                -PI * np.sin(2 * PI * x) * np.sin(PI * y) ** 2)

    def p(self, x, y):
        return np.cos(PI * x) * np.cos(PI * y)

    def f(self, x, y):
        e = self.eta
        lux = 2 * PI ** 3 * np.sin(2 * PI * y) * (2 * np.cos(2 * PI * x) - 1)
        luy = -2 * PI ** 3 * np.sin(2 * PI * x) * (2 * np.cos(2 * PI * y) - 1)
        return (-e * lux - PI * np.sin(PI * x) * np.cos(PI * y),
                -e * luy - PI * np.cos(PI * x) * np.sin(PI * y))


class PolynomialPatch:
    """psi = x^2 (1-x)^2 y^2 (1-y)^2 (u in Q_4^2, zero on the boundary),
    p = (x - 1/2)(y - 1/2)^3 in Q_3, eta = 1.  For k >= 4 both lie in the
    discrete spaces, so SIP consistency makes the discrete solution exact."""

    def __init__(self):
        X = Polynomial([0, 0, 1]) * Polynomial([1, -1]) ** 2
        self.X, self.Y = X, X

    def u(self, x, y):
        X, Y = self.X, self.Y
        return X(x) * Y.deriv()(y), -X.deriv()(x) * Y(y)

    def p(self, x, y):
        return (x - 0.5) * (y - 0.5) ** 3

    def f(self, x, y):
        X, Y = self.X, self.Y
        lux = X.deriv(2)(x) * Y.deriv()(y) + X(x) * Y.deriv(3)(y)
        luy = -(X.deriv(3)(x) * Y(y) + X.deriv()(x) * Y.deriv(2)(y))
        return -lux + (y - 0.5) ** 3, -luy + 3 * (x - 0.5) * (y - 0.5) ** 2
