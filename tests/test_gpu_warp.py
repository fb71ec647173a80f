"""GPU parity of the warp-row FP32 SIP apply (schedule code 6: one thread per
element, one warp per tile row, element blocks staged with asynchronous
16-byte copies) against the FP64 oracle, through the C ABI: the operator
element by element on ragged meshes with every boundary kind and k = 1..5,
sampled element rows of the full-size 512^2 k = 4 and 256^2 k = 5 meshes, and
the FP32 V-cycle run on it (y = alpha A x + beta z, in place where z = y)."""
import numpy as np
import pytest
import torch

from oracle import materials, multigrid, sip
from paper_1607_03777_gb300 import api, synth

pytestmark = pytest.mark.gpu

SINK = synth.SINKER_BC
BCS = [("navier",) * 4, SINK, ("dirichlet",) * 4, ("neumann", "dirichlet", "navier", "neumann")]
TOL32 = 1e-5
WARP = 6


def dev(a, dtype=torch.float64):
    return torch.as_tensor(np.ascontiguousarray(a)).to(device="cuda", dtype=dtype)


def host(t):
    return t.detach().cpu().numpy().astype(np.float64)


def errs(got, ref):
    d = got - ref
    return np.linalg.norm(d) / np.linalg.norm(ref), np.abs(d).max() / np.abs(ref).max()


@pytest.mark.parametrize("k", [1, 2, 3, 4, 5])
@pytest.mark.parametrize("mesh", [(1, 1), (3, 2), (37, 3), (4, 35), (33, 9), (70, 11)])
def test_apply_A_f32_warp(ctx, k, mesh):
    """The FP32 operator against the assembled A applied to the same FP32
    data, element by element: tiles cut by both mesh edges, rows whose first
    element is not 16-byte aligned (odd nx, odd N), halo rows and columns."""
    nx, ny = mesh
    for i, bc in enumerate(BCS):
        eta = synth.random_eta(nx * ny, 1900 + 10 * k + i, (0.0, 3.0))
        prob = api.Problem(ctx, nx, ny, k, eta, bc=bc, lx=1.0, ly=0.7)
        prob.set_schedule(apply=[0, WARP])
        assert prob.schedule()["apply"][1] == WARP
        A = sip.assemble_A(sip.Problem(nx, ny, k, eta, bc=bc, lx=1.0, ly=0.7))
        x32 = synth.random_vector(prob.n_u, seed=170 + i).astype(np.float32)
        y32 = torch.full((prob.n_u,), float("nan"), dtype=torch.float32, device="cuda")
        prob.apply_A_f32(dev(x32, torch.float32), y32)
        got = host(y32)
        assert np.isfinite(got).all(), bc   # every output entry written
        e2, emax = errs(got, A @ x32.astype(np.float64))
        assert e2 < TOL32 and emax < 2 * TOL32, (bc, e2, emax)


@pytest.mark.parametrize("n,k", [(512, 4), (512, 3), (256, 5)])
def test_apply_A_f32_warp_full_size_sampled(ctx, n, k):
    """Full-size FP32 operator (the many-disc 512^2 mesh at k = 4 and 3, a
    256^2 k = 5 box mesh): sampled element rows rebuilt one by one by the
    oracle, corners, edges, tile seams and elements at viscosity jumps."""
    wl = synth.many_discs(k=k) if n == 512 else synth.single_box_inclusion(n=n, k=k)
    eta_d, _ = ctx.rasterise_inclusions(n, n, wl.shapes)
    eta = eta_d.cpu().numpy()
    prob = api.Problem(ctx, n, n, k, eta, bc=wl.bc)
    prob.set_schedule(apply=[0, WARP])
    ref = sip.Problem(n, n, k, eta, bc=wl.bc)
    nb = prob.n_u // (n * n)
    x = synth.random_vector(prob.n_u, seed=15, dtype=np.float32).astype(np.float64)
    y = torch.full((prob.n_u,), float("nan"), dtype=torch.float32, device="cuda")
    prob.apply_A_f32(dev(x, torch.float32), y)
    y = host(y)
    assert np.isfinite(y).all()
    E = eta.reshape(n, n)
    jump = np.argwhere(E != np.roll(E, 1, axis=1))[:4]
    picks = [(0, 0), (n - 1, 0), (0, n - 1), (n - 1, n - 1), (n // 2, 0), (0, n // 3),
             (31, 3), (32, 4), (63, 7), (64, 8), (n - 1, n // 2), (n // 2, n - 1),
             (n // 2 + 1, n // 2 - 3)]
    picks += [(int(c), int(r)) for r, c in jump]
    for ex, ey in picks:
        e = ey * n + ex
        ref_row = np.zeros(nb)
        for f, blk in sip.element_rows_A(ref, ex, ey).items():
            ref_row += blk @ x[f * nb:(f + 1) * nb]
        e2, _ = errs(y[e * nb:(e + 1) * nb], ref_row)
        assert e2 < TOL32, (ex, ey, e2)


@pytest.mark.parametrize("k", [2, 3, 4])
def test_vcycle_f32_warp(ctx, k):
    """The FP32 V-cycle with the warp-row apply and unfused smoother steps
    (residuals r = b - A y and r -= A d in place) against the oracle's
    V-cycle, as the V-cycle of the other FP32 kernels."""
    nx = ny = 16
    eta, _ = materials.rasterise_inclusions(nx, ny, synth.single_box_inclusion(nx, k, 1e3).shapes)
    prob = api.Problem(ctx, nx, ny, k, eta, bc=SINK, n_hlevels=2, seed=9, precision="mixed",
                       mixed_fp64_ratio=0.0)
    prob.set_schedule(apply=[0, WARP], fused=[-1, 0])
    ref = sip.Problem(nx, ny, k, eta, bc=SINK)
    A = sip.assemble_A(ref)
    mg = multigrid.HPMultigrid(ref, A, 2, seed=9)
    r = synth.random_vector(prob.n_u, 78).astype(np.float32)
    z = torch.empty(prob.n_u, dtype=torch.float32, device="cuda")
    prob.vcycle_f32(dev(r, torch.float32), z)
    sched = prob.schedule()
    assert sched["apply"][1] == WARP and sched["fused"][1] == 0, sched
    ref_z = mg(r.astype(np.float64))
    assert np.linalg.norm(host(z) - ref_z) < 2e-4 * np.linalg.norm(ref_z)


def test_warp_code_rejected_for_fp64(ctx):
    """Code 6 exists for the FP32 operator only."""
    prob = api.Problem(ctx, 8, 8, 2, np.ones(64))
    with pytest.raises(api.SipError):
        prob.set_schedule(apply=[6, 6])
