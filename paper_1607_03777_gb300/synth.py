"""Seeded synthetic inputs shaped like the paper's workloads.

This module draws numbers only: inclusion lists, viscosity contrasts,
mesh sizes, request arrival times and random vectors.  It holds none of the
method's arithmetic (no rasterisation, no quadrature, no operator), so both
the CUDA library and the oracle consume exactly the same inputs.

Generators use numpy's PCG64 with the seeds named per workload.

Inclusion records are rows (kind, a, b, c, d, eta_i, rho_i):
kind 0 = disc with centre (a, b) and radius c; kind 1 = box [a, b] x [c, d].
"""
from dataclasses import dataclass, field

import numpy as np

NAVIER, NEUMANN, DIRICHLET = "navier", "neumann", "dirichlet"
SINKER_BC = (NAVIER, NAVIER, NAVIER, NEUMANN)   # Neumann top, Navier elsewhere
GRAVITY = 10.0


@dataclass
class Workload:
    name: str
    nx: int
    ny: int
    k: int
    shapes: np.ndarray            # inclusion records, shape (n, 7)
    bc: tuple = SINKER_BC
    eta_bg: float = 1.0
    rho_bg: float = 1.0
    n_hlevels: int = 0
    rtol: float = 1e-8
    precision: str = "fp64"
    meta: dict = field(default_factory=dict)


def box(xa, xb, ya, yb, eta, rho):
    return np.array([1.0, xa, xb, ya, yb, eta, rho])


def disc(cx, cy, r, eta, rho):
    return np.array([0.0, cx, cy, r, 0.0, eta, rho])


def single_box_inclusion(n=128, k=3, eta_in=1e4, rho_in=1.2, n_hlevels=3):
    """Square inclusion [0.25, 0.75]^2 of viscosity eta_in and density
    rho_in in a unit-viscosity, unit-density medium; Neumann top, Navier
    elsewhere; Q^2_1 coarse space with n_hlevels h-coarsenings."""
    return Workload("single_box_inclusion", n, n, k,
                    np.stack([box(0.25, 0.75, 0.25, 0.75, eta_in, rho_in)]),
                    n_hlevels=n_hlevels, rtol=1e-8,
                    meta={"eta_in": eta_in, "rho_in": rho_in})


def random_discs(n_discs, radius, log10_contrast, seed, rho_in=1.2, shared_eta=False):
    """n_discs discs with centres uniform in the unit square; log10 of the
    disc viscosity uniform in log10_contrast = (lo, hi) (one value for all
    discs when shared_eta)."""
    g = np.random.Generator(np.random.PCG64(seed))
    c = g.uniform(0.0, 1.0, size=(n_discs, 2))
    lo, hi = log10_contrast
    if shared_eta:
        le = np.full(n_discs, g.uniform(lo, hi))
    else:
        le = g.uniform(lo, hi, size=n_discs)
    return np.stack([disc(c[i, 0], c[i, 1], radius, 10.0 ** le[i], rho_in) for i in range(n_discs)])


def many_discs(n=512, k=4, n_discs=64, radius=0.02, seed=3, precision="mixed", n_hlevels=5):
    """64 discs of radius 0.02 at seeded random centres, log10(eta) ~ U[0, 6]."""
    return Workload("many_discs", n, n, k, random_discs(n_discs, radius, (0.0, 6.0), seed),
                    n_hlevels=n_hlevels, rtol=1e-8, precision=precision)


# centres and radii of the six sedimenting inclusions of Sec. 7.3
SINKERS = [(0.84, 0.39, 0.089), (0.79, 0.91, 0.059), (0.33, 0.76, 0.063),
           (0.55, 0.47, 0.081), (0.14, 0.60, 0.05), (0.24, 0.13, 0.09)]


def six_sinkers(n=64, k=2, eta_in=1e3, n_hlevels=2):
    """The six sedimenting circular inclusions of Sec. 7.3 (positions and
    radii as listed there), density 1.2 against 1."""
    return Workload("six_sinkers", n, n, k,
                    np.stack([disc(a, b, r, eta_in, 1.2) for a, b, r in SINKERS]),
                    n_hlevels=n_hlevels, rtol=1e-6)


def jittered_sinkers(seed, log10_contrast, jitter=0.02, rho_in=1.2):
    """The six inclusions of Sec. 7.3 with every centre moved by
    U[-jitter, jitter] in x and y, all of one viscosity 10^U[lo, hi]."""
    g = np.random.Generator(np.random.PCG64(seed))
    le = g.uniform(*log10_contrast)
    out = []
    for a, b, r in SINKERS:
        dx, dy = g.uniform(-jitter, jitter, size=2)
        out.append(disc(a + dx, b + dy, r, 10.0 ** le, rho_in))
    return np.stack(out)


def batch_instances(count=128, seed=4, log10_contrast=(2.0, 6.0)):
    """Independent instances: side uniform in {32, 64, 128, 256}, k uniform
    in {2, 3, 4, 5}, the six inclusions of Sec. 7.3 with jittered centres
    and one contrast 10^U[2,6] (above 1e5 the 1e-8 relative residual lies
    below what an FP64 residual can resolve on these meshes: the solves
    use iterative refinement with a double-double residual)."""
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(g.choice([32, 64, 128, 256]))
        k = int(g.choice([2, 3, 4, 5]))
        sub = int(g.integers(0, 2 ** 31))
        shapes = jittered_sinkers(sub, log10_contrast)
        out.append(Workload(f"batch_{i}", n, n, k, shapes, n_hlevels=levels_to_17(n),
                            rtol=1e-8, precision="mixed"))
    return out


def checkerboard(n=64, k=2, eta_hi=1e6, n_hlevels=3):
    """A 2 x 2 viscosity checkerboard on the unit square (the SolCx jump at
    x = 1/2 plus one at y = 1/2, Sec. 7.2): eta_hi in the lower-left and
    upper-right quadrants, 1 elsewhere, Navier on every side.  The paper's
    SolCx forcing is only cited, so the flow is driven by a disc of density
    1.2 (unit viscosity) at (0.3, 0.65), radius 0.1, inside the upper-left
    quadrant; its sinking crosses both jumps."""
    shapes = np.stack([box(0.0, 0.5, 0.0, 0.5, eta_hi, 1.0),
                       box(0.5, 1.0, 0.5, 1.0, eta_hi, 1.0),
                       disc(0.3, 0.65, 0.1, 1.0, 1.2)])
    return Workload("checkerboard", n, n, k, shapes, bc=(NAVIER,) * 4, n_hlevels=n_hlevels,
                    rtol=1e-6, meta={"eta_hi": eta_hi})


def levels_to_17(n):
    """Number of h-coarsenings that brings an n-element side down to 16
    elements (17 vertices), the coarsest grid the paper keeps."""
    lv = 0
    while n % 2 == 0 and n > 16:
        n //= 2
        lv += 1
    return lv


def request_stream(count=2000, rate=200.0, seed=5, log10_contrast=(0.0, 6.0)):
    """Poisson arrivals at ``rate`` per second; side log-uniform in
    [32, 512] rounded to a multiple of 16; k in {2..6}; the six jittered
    inclusions of Sec. 7.3 with one contrast 10^U[0,6].  Returns
    (arrival_times, workloads)."""
    g = np.random.Generator(np.random.PCG64(seed))
    gaps = g.exponential(1.0 / rate, size=count)
    t = np.cumsum(gaps)
    wl = []
    for i in range(count):
        side = int(np.exp(g.uniform(np.log(32), np.log(512))))
        side = max(32, min(512, 16 * int(round(side / 16))))
        k = int(g.integers(2, 7))
        sub = int(g.integers(0, 2 ** 31))
        shapes = jittered_sinkers(sub, log10_contrast)
        wl.append(Workload(f"req_{i}", side, side, k, shapes, n_hlevels=levels_to_17(side),
                           rtol=1e-8, precision="mixed"))
    return t, wl


def random_vector(n, seed, dtype=np.float64):
    """Standard normal test vector."""
    return np.random.Generator(np.random.PCG64(seed)).standard_normal(n).astype(dtype)


def random_eta(ne, seed, log10_range=(0.0, 3.0)):
    """Element viscosities 10^U[lo, hi] for operator tests."""
    g = np.random.Generator(np.random.PCG64(seed))
    return 10.0 ** g.uniform(*log10_range, size=ne)
