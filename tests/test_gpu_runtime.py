"""Batched and served solves: every result equals the same solve run alone
(through the C ABI), admission by device footprint, request bookkeeping."""
import numpy as np
import pytest
import torch

from paper_1607_03777_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu


def _instances(count, seed):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(g.choice([16, 32]))
        k = int(g.choice([2, 3]))
        shapes = synth.random_discs(4, 0.08, (1.0, 3.0), int(g.integers(0, 2 ** 31)), shared_eta=True)
        out.append((n, k, shapes, "mixed" if i % 2 else "fp64"))
    return out


def _alone(ctx, n, k, shapes, precision):
    eta, rho = ctx.rasterise_inclusions(n, n, shapes)
    prob = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=synth.SINKER_BC,
                       n_hlevels=synth.levels_to_17(n) if n > 16 else 1, seed=2,
                       precision=precision)
    f = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    prob.rhs_body_force(rho, synth.GRAVITY, f)
    u = torch.empty_like(f)
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    rep = prob.solve(f, u, p, rtol=1e-8)
    return prob, f, u, p, rep, eta.cpu().numpy(), rho.cpu().numpy()


def test_batch_matches_alone(ctx):
    inst = _instances(6, 1)
    alone = [_alone(ctx, *x) for x in inst]
    probs = [a[0] for a in alone]
    fs = [a[1] for a in alone]
    us = [torch.empty_like(a[2]) for a in alone]
    ps = [torch.empty_like(a[3]) for a in alone]
    st, reps = api.solve_batch(ctx, probs, fs, us, ps, n_streams=4, rtol=1e-8)
    assert st == _lib.SIP_OK
    for a, u, p, r in zip(alone, us, ps, reps):
        assert r["status"] == 0 and r["rel_residual"] <= 1e-8
        assert torch.equal(u, a[2]) and torch.equal(p, a[3])


def test_server_matches_alone_and_reports_latency(ctx):
    inst = _instances(8, 2)
    alone = [_alone(ctx, *x) for x in inst]
    srv = api.Server(ctx, budget_bytes=8 << 30, max_slots=3)
    outs = {}
    for rid, (x, a) in enumerate(zip(inst, alone)):
        n, k, shapes, precision = x
        st, u, p = srv.submit(rid, n, n, k, a[5], a[6], g=synth.GRAVITY, bc=synth.SINKER_BC,
                              n_hlevels=synth.levels_to_17(n) if n > 16 else 1, seed=2,
                              precision=precision)
        assert st == _lib.SIP_OK
        outs[rid] = (u, p)
    srv.drain()
    done = dict(srv.poll())
    assert sorted(done) == list(range(len(inst)))
    for rid, a in enumerate(alone):
        rep = done[rid]
        assert rep["status"] == 0 and rep["rel_residual"] <= 1e-8
        assert rep["solve_ms"] > 0
        u, p = outs[rid]
        assert np.array_equal(u, a[2].cpu().numpy()) and np.array_equal(p, a[3].cpu().numpy())
    assert srv.stats() == {"queued": 0, "running": 0, "bytes_in_use": 0}
    srv.close()


def test_server_admission_rejects_oversized_request(ctx):
    n, k = 32, 3
    need = api.footprint(ctx, nx=n, ny=n, k=k, eta=np.ones(n * n), n_hlevels=1)
    assert need > 0
    srv = api.Server(ctx, budget_bytes=need // 2, max_slots=2)
    st, _, _ = srv.submit(7, n, n, k, np.ones(n * n), np.ones(n * n), n_hlevels=1)
    assert st == 7     # SIP_ERR_REJECTED
    got = srv.poll()
    assert got and got[0][0] == 7 and got[0][1]["status"] == 7
    srv.close()


def test_server_queues_beyond_slots(ctx):
    """More requests than slots: all are admitted in turn and finish."""
    srv = api.Server(ctx, budget_bytes=8 << 30, max_slots=1)
    n, k = 16, 2
    eta = synth.random_eta(n * n, 3, (0.0, 2.0))
    for rid in range(4):
        srv.submit(rid, n, n, k, eta, np.ones(n * n), n_hlevels=1, bc=synth.SINKER_BC)
    srv.drain()
    done = srv.poll()
    assert sorted(i for i, _ in done) == [0, 1, 2, 3]
    assert all(r["status"] == 0 for _, r in done)
    srv.close()


@pytest.mark.parametrize("k,precision", [(2, "fp64"), (3, "mixed"), (5, "fp64"), (6, "fp64")])
def test_autotuned_schedule(ctx, k, precision):
    """The first set-up of a shape picks its kernels by timing; a second
    problem of the same shape reuses the choice; the schedule holds only
    kernels that exist for the degree (fused smoother steps up to degree 3,
    element kernels up to degree 5, the tile kernel alone above)."""
    n = 48
    shapes = synth.jittered_sinkers(3, (2.0, 2.0))
    a = _alone(ctx, n, k, shapes, precision)
    b = _alone(ctx, n, k, shapes, precision)
    sa, sb = a[0].schedule(), b[0].schedule()
    assert sa == sb
    if k <= 5:
        assert all(v in (1, 2, 3) for v in sa["apply"])
    else:
        assert sa["apply"] == [3, 3]
    if k <= 3:
        assert all(v in (0, 1) for v in sa["fused"])
    else:
        assert sa["fused"] == [0, 0]
    # same shape, same kernels: bit-identical solves
    assert torch.equal(a[2], b[2]) and torch.equal(a[3], b[3])


def test_batch_allocates_then_problems_destroyed(ctx):
    """Problems whose solver workspace is first allocated inside a batched
    solve (on the batch's worker streams) are solved again alone and then
    destroyed after the batch has returned."""
    inst = _instances(4, 7)
    probs, fs, us, ps = [], [], [], []
    for n, k, shapes, precision in inst:
        eta, rho = ctx.rasterise_inclusions(n, n, shapes)
        prob = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=synth.SINKER_BC,
                           n_hlevels=synth.levels_to_17(n) if n > 16 else 1, seed=2,
                           precision=precision)
        f = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        prob.rhs_body_force(rho, synth.GRAVITY, f)
        probs.append(prob)
        fs.append(f)
        us.append(torch.empty_like(f))
        ps.append(torch.empty(prob.n_p, dtype=torch.float64, device="cuda"))
    st, reps = api.solve_batch(ctx, probs, fs, us, ps, n_streams=4, rtol=1e-8)
    assert st == 0 and all(r["status"] == 0 for r in reps)
    u2 = torch.empty_like(us[0])
    p2 = torch.empty_like(ps[0])
    probs[0].solve(fs[0], u2, p2, rtol=1e-8)
    assert torch.equal(u2, us[0])
    for pr in probs:
        pr.close()
    torch.cuda.synchronize()


def test_batch_with_refinement_matches_alone(ctx):
    """Iterative refinement through the batched path: each instance, solved
    with refine = 4 to 1e-10 alongside the others, equals the same refined
    solve run alone, bit for bit, and reports its correction solves; invalid
    options are refused before any work."""
    inst = _instances(4, 3)
    alone = []
    for n, k, shapes, precision in inst:
        prob, f, _, _, _, _, _ = _alone(ctx, n, k, shapes, precision)
        u = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
        p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
        rep = prob.solve(f, u, p, rtol=1e-10, refine=4)
        assert rep["refine_steps"] >= 1 and rep["rel_residual"] <= 1e-10, rep
        alone.append((prob, f, u, p))
    us = [torch.empty_like(a[2]) for a in alone]
    ps = [torch.empty_like(a[3]) for a in alone]
    st, reps = api.solve_batch(ctx, [a[0] for a in alone], [a[1] for a in alone], us, ps,
                               n_streams=2, rtol=1e-10, refine=4)
    assert st == _lib.SIP_OK
    for a, u, p, r in zip(alone, us, ps, reps):
        assert r["status"] == 0 and r["refine_steps"] >= 1
        assert torch.equal(u, a[2]) and torch.equal(p, a[3])
    st, _ = api.solve_batch(ctx, [a[0] for a in alone], [a[1] for a in alone], us, ps,
                            refine=101)
    assert _lib.STATUS_NAMES[st] == "SIP_ERR_INVALID_ARG"
