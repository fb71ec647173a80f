"""Batched and served solves: every result equals the same solve run alone
(through the C ABI) and meets the tolerance by the FP64 oracle's own
assembled matrices; admission by device footprint, request bookkeeping,
deadlines, cancellation and rejected inputs."""
import numpy as np
import pytest
import torch

from oracle import krylov, sip
from paper_1607_03777_gb300 import _lib, api, synth

pytestmark = pytest.mark.gpu


def _instances(count, seed, kmax=3, log_contrast=(1.0, 3.0)):
    g = np.random.Generator(np.random.PCG64(seed))
    out = []
    for i in range(count):
        n = int(g.choice([16, 32]))
        k = int(g.integers(2, kmax + 1))
        shapes = synth.random_discs(4, 0.08, log_contrast, int(g.integers(0, 2 ** 31)),
                                    shared_eta=True)
        out.append((n, k, shapes, "mixed" if i % 2 else "fp64"))
    return out


def _oracle_residual(n, k, eta, rho, u, p):
    """||b - K x|| / ||b|| of a result with the oracle's assembled A, B and
    load vector (FP64, independent of the CUDA path)."""
    ref = sip.Problem(n, n, k, eta, bc=synth.SINKER_BC)
    f = sip.rhs_body_force(ref, rho, g=synth.GRAVITY)
    K = krylov.stokes_matrix(sip.assemble_A(ref), sip.assemble_B(ref)).tocsr()
    b = np.concatenate([f, np.zeros(ref.num.n_p)])
    x = np.concatenate([np.asarray(u, dtype=np.float64), np.asarray(p, dtype=np.float64)])
    return np.linalg.norm(b - K @ x) / np.linalg.norm(b)


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
    """Degrees 2..5, contrasts 10^U[1, 5]: batched = alone bit for bit, and
    the oracle's residual of every result meets 1e-8."""
    inst = _instances(8, 1, kmax=5, log_contrast=(1.0, 5.0))
    alone = [_alone(ctx, *x) for x in inst]
    probs = [a[0] for a in alone]
    fs = [a[1] for a in alone]
    us = [torch.empty_like(a[2]) for a in alone]
    ps = [torch.empty_like(a[3]) for a in alone]
    st, reps = api.solve_batch(ctx, probs, fs, us, ps, n_streams=4, rtol=1e-8)
    assert st == _lib.SIP_OK
    for x, a, u, p, r in zip(inst, alone, us, ps, reps):
        assert r["status"] == 0 and r["rel_residual"] <= 1e-8
        assert torch.equal(u, a[2]) and torch.equal(p, a[3])
        res = _oracle_residual(x[0], x[1], a[5], a[6], u.cpu().numpy(), p.cpu().numpy())
        assert res <= 1.05e-8, (x[:2], x[3], res)


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_batch_grouped_matches_alone_and_oracle(ctx, precision):
    """Instances of one precision: the inner solves of the whole group run
    as one batched graph (one launch per stage and degree for all
    instances).  Every result meets 1e-8 by the oracle's own matrices and
    agrees with the same solve run alone (same arithmetic, another blocking
    of the dot products) to 1e-5."""
    g = np.random.Generator(np.random.PCG64(11))
    inst = []
    for _ in range(6):
        n = int(g.choice([16, 32]))
        k = int(g.integers(2, 6))
        shapes = synth.random_discs(4, 0.08, (1.0, 4.0), int(g.integers(0, 2 ** 31)),
                                    shared_eta=True)
        inst.append((n, k, shapes, precision))
    alone = [_alone(ctx, *x) for x in inst]
    us = [torch.empty_like(a[2]) for a in alone]
    ps = [torch.empty_like(a[3]) for a in alone]
    st, reps = api.solve_batch(ctx, [a[0] for a in alone], [a[1] for a in alone], us, ps,
                               n_streams=len(inst), rtol=1e-8, grouped=True)
    assert st == _lib.SIP_OK, reps
    for x, a, u, p, r in zip(inst, alone, us, ps, reps):
        assert r["status"] == 0 and r["rel_residual"] <= 1e-8, (x[:2], r)
        res = _oracle_residual(x[0], x[1], a[5], a[6], u.cpu().numpy(), p.cpu().numpy())
        assert res <= 1.05e-8, (x[:2], res)
        du = float(torch.linalg.norm(u - a[2]) / torch.linalg.norm(a[2]))
        assert du <= 1e-5, (x[:2], du)
    # a group must share one precision
    mixed_probs = [alone[0][0], _alone(ctx, 16, 2, inst[0][2],
                                       "fp64" if precision == "mixed" else "mixed")[0]]
    st, _ = api.solve_batch(ctx, mixed_probs, [alone[0][1], alone[0][1]][:1] +
                            [torch.zeros(mixed_probs[1].n_u, dtype=torch.float64, device="cuda")],
                            [torch.empty_like(us[0]), torch.empty(mixed_probs[1].n_u,
                                                                  dtype=torch.float64,
                                                                  device="cuda")],
                            [torch.empty_like(ps[0]), torch.empty(mixed_probs[1].n_p,
                                                                  dtype=torch.float64,
                                                                  device="cuda")],
                            grouped=True)
    assert _lib.STATUS_NAMES[st] == "SIP_ERR_INVALID_ARG"


def test_server_matches_alone_and_reports_latency(ctx):
    inst = _instances(8, 2, kmax=5, log_contrast=(1.0, 5.0))
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
        n, k = inst[rid][:2]
        assert _oracle_residual(n, k, a[5], a[6], u, p) <= 1.05e-8, inst[rid][:2]
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


def test_server_backfills_past_a_large_head(ctx):
    """A large request that does not fit the free budget does not hold up the
    small requests queued behind it: with one large solve running and a
    second large one at the head of the queue, the small ones run in the
    spare memory and finish first; the second large one still runs."""
    nb, ns = 128, 16
    eta_b = synth.random_eta(nb * nb, 5, (0.0, 2.0))
    eta_s = synth.random_eta(ns * ns, 6, (0.0, 2.0))
    big = api.footprint(ctx, nx=nb, ny=nb, k=3, eta=eta_b, n_hlevels=3)
    small = api.footprint(ctx, nx=ns, ny=ns, k=2, eta=eta_s, n_hlevels=1)
    assert small < big // 2
    srv = api.Server(ctx, budget_bytes=big + 3 * small // 2, max_slots=2)
    order = [("big", 0), ("big", 1), ("small", 2), ("small", 3)]
    for kind, rid in order:
        if kind == "big":
            st, _, _ = srv.submit(rid, nb, nb, 3, eta_b, np.ones(nb * nb), n_hlevels=3,
                                  bc=synth.SINKER_BC)
        else:
            st, _, _ = srv.submit(rid, ns, ns, 2, eta_s, np.ones(ns * ns), n_hlevels=1,
                                  bc=synth.SINKER_BC)
        assert st == _lib.SIP_OK
    srv.drain()
    done = srv.poll()
    ids = [i for i, _ in done]
    assert sorted(ids) == [0, 1, 2, 3]
    assert all(r["status"] == 0 and r["rel_residual"] <= 1e-8 for _, r in done)
    assert ids.index(2) < ids.index(1) and ids.index(3) < ids.index(1), ids
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
        assert all(v in (1, 2, 3, 4, 5) for v in sa["apply"])
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


# ------------------------------------------------------------ failure paths
def _box_problem(ctx, n=32, k=3, precision="fp64"):
    wl = synth.single_box_inclusion(n=n, k=k, eta_in=1e3, n_hlevels=1)
    eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
    prob = api.Problem(ctx, n, n, k, eta.cpu().numpy(), bc=wl.bc, n_hlevels=1, seed=1,
                       precision=precision)
    f = torch.empty(prob.n_u, dtype=torch.float64, device="cuda")
    prob.rhs_body_force(rho, synth.GRAVITY, f)
    return prob, f, eta.cpu().numpy(), rho.cpu().numpy()


def test_solve_rejects_non_finite_load(ctx):
    """A NaN or infinite entry in f is refused (SIP_ERR_INVALID_ARG) before
    any Krylov work, and the library stays usable."""
    prob, f, _, _ = _box_problem(ctx)
    u = torch.empty_like(f)
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    for bad in (float("nan"), float("inf")):
        g = f.clone()
        g[17] = bad
        rep = prob.solve(g, u, p, rtol=1e-8, check=False)
        assert _lib.STATUS_NAMES[rep["status"]] == "SIP_ERR_INVALID_ARG", rep
    rep = prob.solve(f, u, p, rtol=1e-8)
    assert rep["status"] == 0


@pytest.mark.parametrize("outer", ["fgmres", "gcr"])
def test_solve_time_limit(ctx, outer):
    """A time limit shorter than one outer iteration stops the solve after
    that iteration with SIP_ERR_TIMEOUT; u, p hold the finite last iterate;
    the same problem then solves normally."""
    prob, f, _, _ = _box_problem(ctx)
    u = torch.empty_like(f)
    p = torch.empty(prob.n_p, dtype=torch.float64, device="cuda")
    prob.solve(f, u, p, rtol=1e-8, outer_krylov=outer)   # set-up outside the limit
    rep = prob.solve(f, u, p, rtol=1e-8, time_limit_ms=1e-3, outer_krylov=outer, check=False)
    assert _lib.STATUS_NAMES[rep["status"]] == "SIP_ERR_TIMEOUT", rep
    assert 1 <= rep["outer_its"] <= 2 and 0.0 < rep["rel_residual"] < 1.0
    assert torch.isfinite(u).all() and torch.isfinite(p).all()
    rep = prob.solve(f, u, p, rtol=1e-8, outer_krylov=outer)
    assert rep["status"] == 0


def test_server_deadline_cancel_and_bad_input(ctx):
    """One slot, requests queued behind a running one: a request whose
    deadline passes while it waits is reported SIP_ERR_TIMEOUT unsolved; a
    queued request that is cancelled is reported SIP_ERR_CANCELLED; ids that
    are neither queued nor running cannot be cancelled; non-finite inputs are
    refused at submission; the others finish normally."""
    n, k = 64, 3
    wl = synth.single_box_inclusion(n=n, k=k, eta_in=1e3, n_hlevels=2)
    eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
    eta, rho = eta.cpu().numpy(), rho.cpu().numpy()
    srv = api.Server(ctx, budget_bytes=8 << 30, max_slots=1)
    kw = dict(bc=wl.bc, n_hlevels=2, seed=1)
    assert srv.submit(0, n, n, k, eta, rho, **kw)[0] == 0            # runs first
    assert srv.submit(1, n, n, k, eta, rho, opts={"time_limit_ms": 1e-3}, **kw)[0] == 0
    assert srv.submit(2, n, n, k, eta, rho, **kw)[0] == 0
    assert srv.cancel(2) == 0
    assert srv.submit(3, n, n, k, eta, rho, **kw)[0] == 0
    assert _lib.STATUS_NAMES[srv.cancel(99)] == "SIP_ERR_INVALID_ARG"
    bad = rho.copy()
    bad[5] = float("nan")
    assert _lib.STATUS_NAMES[srv.submit(4, n, n, k, eta, bad, **kw)[0]] == "SIP_ERR_INVALID_ARG"
    neg = eta.copy()
    neg[3] = -1.0
    assert _lib.STATUS_NAMES[srv.submit(5, n, n, k, neg, rho, **kw)[0]] == "SIP_ERR_INVALID_ARG"
    srv.drain()
    done = dict(srv.poll())
    assert sorted(done) == [0, 1, 2, 3]
    names = {i: _lib.STATUS_NAMES[r["status"]] for i, r in done.items()}
    assert names == {0: "SIP_OK", 1: "SIP_ERR_TIMEOUT", 2: "SIP_ERR_CANCELLED", 3: "SIP_OK"}
    assert _lib.STATUS_NAMES[srv.cancel(0)] == "SIP_ERR_INVALID_ARG"   # finished
    assert srv.stats() == {"queued": 0, "running": 0, "bytes_in_use": 0}
    srv.close()


def test_server_cancel_running_request(ctx):
    """Cancelling a running request stops it at its next outer iteration:
    reported SIP_ERR_CANCELLED well before the uncancelled solve would end."""
    import time
    n, k = 256, 4
    wl = synth.single_box_inclusion(n=n, k=k, eta_in=1e4, n_hlevels=4)
    eta, rho = ctx.rasterise_inclusions(n, n, wl.shapes)
    eta, rho = eta.cpu().numpy(), rho.cpu().numpy()
    srv = api.Server(ctx, budget_bytes=16 << 30, max_slots=1)
    t0 = time.perf_counter()
    srv.submit(0, n, n, k, eta, rho, bc=wl.bc, n_hlevels=4, seed=1)
    for _ in range(2000):                 # wait until it runs (bounded)
        if srv.stats()["running"] == 1:
            break
        time.sleep(0.005)
    time.sleep(0.05)
    assert srv.cancel(0) == 0
    srv.drain()
    (rid, rep), = srv.poll()
    assert rid == 0 and _lib.STATUS_NAMES[rep["status"]] == "SIP_ERR_CANCELLED", rep
    assert rep["outer_its"] >= 1
    srv.close()
