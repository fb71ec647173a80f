"""GPU parity of the operator kernels (A, A_f32, B, B^T, load vector,
rasterisation) against the FP64 oracle, through the C ABI.

Tolerances (relative, 2-norm and element-wise max against the max entry):
FP64 apply 1e-10, FP32 apply 1e-5; integer-valued decisions bit-exact.
"""
import numpy as np
import pytest
import torch

from oracle import materials, sip
from paper_1607_03777_gb300 import api, synth

pytestmark = pytest.mark.gpu

BCS = [("navier",) * 4, ("navier", "navier", "navier", "neumann"),
       ("dirichlet",) * 4, ("neumann", "dirichlet", "navier", "neumann")]
MESHES = [(1, 1), (3, 2), (37, 3), (4, 35)]
TOL64, TOL32 = 1e-10, 1e-5


def rel_err(got, ref, mag=None):
    """Relative 2-norm and max-entry errors.  ``mag`` (the natural output
    scale ||M|| |x| of the operator) guards the denominator when the exact
    result cancels to (near) zero, e.g. B applied to the constant pressure."""
    got = np.asarray(got, dtype=np.float64)
    ref = np.asarray(ref, dtype=np.float64)
    floor2 = np.linalg.norm(mag) if mag is not None else 1e-300
    floorm = np.abs(mag).max() if mag is not None else 1e-300
    return (np.linalg.norm(got - ref) / max(np.linalg.norm(ref), floor2),
            np.abs(got - ref).max() / max(np.abs(ref).max(), floorm))


def make(ctx, nx, ny, k, bc, seed, contrast=3.0, lx=1.0, ly=1.0):
    eta = synth.random_eta(nx * ny, seed, (0.0, contrast))
    prob = api.Problem(ctx, nx, ny, k, eta, bc=bc, lx=lx, ly=ly)
    ref = sip.Problem(nx, ny, k, eta, bc=bc, lx=lx, ly=ly)
    return prob, ref


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("mesh", MESHES)
def test_apply_A_fp64(ctx, k, mesh):
    nx, ny = mesh
    for i, bc in enumerate(BCS):
        prob, ref = make(ctx, nx, ny, k, bc, seed=100 * k + i, lx=1.0, ly=0.7)
        A = sip.assemble_A(ref)
        x = synth.random_vector(prob.n_u, seed=7 + i)
        y = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        prob.apply_A(dev(x), y)
        e2, emax = rel_err(y.cpu().numpy(), A @ x)
        assert e2 < TOL64 and emax < TOL64, (bc, e2, emax)


@pytest.mark.parametrize("k", [1, 3, 4, 6])
@pytest.mark.parametrize("mesh", [(3, 2), (37, 3)])
def test_apply_A_fp32(ctx, k, mesh):
    nx, ny = mesh
    for i, bc in enumerate(BCS):
        prob, ref = make(ctx, nx, ny, k, bc, seed=300 + 10 * k + i)
        A = sip.assemble_A(ref)
        x32 = synth.random_vector(prob.n_u, seed=11 + i, dtype=np.float32)
        y = torch.empty(prob.n_u, dtype=torch.float32, device="cuda")
        prob.apply_A_f32(dev(x32, torch.float32), y)
        e2, emax = rel_err(y.cpu().numpy(), A @ x32.astype(np.float64))
        assert e2 < TOL32 and emax < 2 * TOL32, (bc, e2, emax)


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5, 6])
@pytest.mark.parametrize("mesh", [(1, 1), (3, 2), (5, 4)])
def test_apply_B_and_Bt(ctx, k, mesh):
    nx, ny = mesh
    for i, bc in enumerate(BCS):
        prob, ref = make(ctx, nx, ny, k, bc, seed=500 + k + i, lx=0.8, ly=1.3)
        B = sip.assemble_B(ref)
        xp = synth.random_vector(prob.n_p, seed=21 + i)
        xu = synth.random_vector(prob.n_u, seed=31 + i)
        yu = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        yp = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
        prob.apply_B(dev(xp), yu)
        prob.apply_Bt(dev(xu), yp)
        # the natural scale of B is h |x| (B entries ~ h on the orthonormal
        # basis); it guards cases where the exact result cancels to zero
        # (one Navier element with k = 1: B p = 0 for the constant p)
        h = max(0.8 / nx, 1.3 / ny)
        e2, emax = rel_err(yu.cpu().numpy(), B @ xp, np.full(prob.n_u, h * np.abs(xp).max()))
        assert e2 < TOL64 and emax < TOL64, ("B", bc, e2, emax)
        e2, emax = rel_err(yp.cpu().numpy(), B.T @ xu, np.full(prob.n_p, h * np.abs(xu).max()))
        assert e2 < TOL64 and emax < TOL64, ("Bt", bc, e2, emax)


@pytest.mark.parametrize("k", [1, 4])
def test_rhs_body_force(ctx, k):
    nx, ny = 6, 5
    prob, ref = make(ctx, nx, ny, k, BCS[1], seed=3, lx=2.0, ly=1.0)
    rho = 1.0 + synth.random_eta(nx * ny, 9, (0.0, 0.3))
    f = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    prob.rhs_body_force(dev(rho), 10.0, f)
    e2, emax = rel_err(f.cpu().numpy(), sip.rhs_body_force(ref, rho, g=10.0))
    assert e2 < 1e-14 and emax < 1e-14


@pytest.mark.parametrize("n", [7, 64, 129])
def test_rasterise_bit_exact(ctx, n):
    shapes = np.concatenate([synth.random_discs(40, 0.037, (0.0, 6.0), seed=n),
                             np.stack([synth.box(0.25, 0.75, 0.25, 0.75, 1e4, 1.2)])])
    eta, rho = ctx.rasterise_inclusions(n, n + 3, shapes)
    e_ref, r_ref = materials.rasterise_inclusions(n, n + 3, shapes)
    assert np.array_equal(eta.cpu().numpy(), e_ref)
    assert np.array_equal(rho.cpu().numpy(), r_ref)


def test_rasterise_empty_list(ctx):
    eta, rho = ctx.rasterise_inclusions(5, 3, np.zeros((0, 7)), eta_bg=2.0, rho_bg=0.5)
    assert (eta.cpu().numpy() == 2.0).all() and (rho.cpu().numpy() == 0.5).all()


@pytest.mark.parametrize("n,k,dtype", [(128, 3, "f64"), (512, 4, "f32"), (512, 4, "f64"),
                                       (256, 5, "f32"), (256, 5, "f64")])
def test_apply_A_full_size_sampled(ctx, n, k, dtype):
    """Full-size operator (the single-inclusion 128^2 k=3 and the 512^2 k=4
    many-disc workloads, and a 256^2 k=5 inclusion mesh): sampled element
    rows rebuilt one by one by the oracle, including corners, edges and
    elements at the viscosity jumps."""
    wl = synth.many_discs() if n == 512 else synth.single_box_inclusion(n=n, k=k)
    eta_d, _ = ctx.rasterise_inclusions(n, n, wl.shapes)
    eta = eta_d.cpu().numpy()
    prob = api.Problem(ctx, n, n, k, eta, bc=wl.bc)
    ref = sip.Problem(n, n, k, eta, bc=wl.bc)
    nb = prob.n_u // (n * n)
    if dtype == "f64":
        x = synth.random_vector(prob.n_u, seed=5)
        y = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        prob.apply_A(dev(x), y)
        tol = TOL64
    else:
        x = synth.random_vector(prob.n_u, seed=5, dtype=np.float32).astype(np.float64)
        y = torch.empty(prob.n_u, dtype=torch.float32, device="cuda")
        prob.apply_A_f32(dev(x, torch.float32), y)
        tol = TOL32
    y = y.cpu().numpy().astype(np.float64)
    E = eta.reshape(n, n)
    jump = np.argwhere(E != np.roll(E, 1, axis=1))[:4]
    picks = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (n // 2, 0), (0, n // 3),
             (n - 1, n // 2), (n // 2, n - 1), (n // 2 + 1, n // 2 - 3)]
    picks += [(int(c), int(r)) for r, c in jump]
    for ex, ey in picks:
        e = ey * n + ex
        ref_row = np.zeros(nb)
        for f, blk in sip.element_rows_A(ref, ex, ey).items():
            ref_row += blk @ x[f * nb:(f + 1) * nb]
        e2, emax = rel_err(y[e * nb:(e + 1) * nb], ref_row)
        assert e2 < tol, (ex, ey, e2)


def test_invalid_arguments(ctx):
    with pytest.raises(api.SipError):
        api.Problem(ctx, 4, 4, 7, np.ones(16))
    with pytest.raises(api.SipError):
        api.Problem(ctx, 4, 4, 2, -np.ones(16))
    with pytest.raises(api.SipError):
        api.Problem(ctx, 4, 4, 2, np.full(16, np.nan))
    with pytest.raises(api.SipError):
        api.Problem(ctx, 6, 6, 2, np.ones(36), n_hlevels=2)
