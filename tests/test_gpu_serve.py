"""The continuous-batching request loop: results alone equal results in the mix, admission."""
import time

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import gpu_problem, oracle_qp

pytestmark = pytest.mark.gpu


def _wait(ctx, ticket, n, p, timeout=60.0):
    t0 = time.time()
    while time.time() - t0 < timeout:
        r = ctx.poll(ticket, n, p)
        if r is not None:
            return r
        time.sleep(1e-4)
    raise TimeoutError(ticket)


def test_served_equals_alone():
    from paper_1504_05708_gb300 import duquad as D
    ctx = D.Context(0)
    sizes = [(16, 10.0, 0, 11), (64, 300.0, 1, 12), (200, 2e3, 2, 13), (512, 1e4, 3, 14), (33, 50.0, 1, 15)]
    insts = [W.uneven_instance(*s) for s in sizes]
    probs = [gpu_problem(ctx, i, D.FP32) for i in insts]
    rng = np.random.default_rng(0)
    reqs = []
    for k in range(40):
        j = int(rng.integers(len(insts)))
        q = rng.standard_normal(insts[j].n)
        reqs.append((j, q))
    o = lambda inst: D.opts(inst.alg, eps_out=1e-3, engine=D.ENGINE_CTA)
    # alone: one dq_solve per request
    alone = []
    for j, q in reqs:
        probs[j].set_vectors(q=q)
        xl, xa, lm, (r,) = probs[j].solve(o(insts[j]))
        alone.append((xl.copy(), xa.copy(), r.outer_iters, r.inner_iters))
    for j, i in enumerate(insts):  # restore the original q on the handles
        probs[j].set_vectors(q=i.q)
    ctx.serve_start(slots=64, hbm_budget_bytes=8 << 30)
    try:
        tickets = [(ctx.submit(probs[j], o(insts[j]), q=q), j) for j, q in reqs]
        for (t, j), (xl, xa, oi, ii) in zip(tickets, alone):
            st, sl, sa, sm, r = _wait(ctx, t, insts[j].n, insts[j].p)
            assert st == 0
            assert np.array_equal(sl, xl) and np.array_equal(sa, xa)
            assert (r.outer_iters, r.inner_iters) == (oi, ii)
    finally:
        ctx.serve_stop()
    ctx.close()


def test_served_result_is_eps_optimal():
    from paper_1504_05708_gb300 import duquad as D
    from oracle.kkt import solve_kkt
    ctx = D.Context(0)
    inst = W.single_dense(n=10, p=5, seed=3, g_scale=0.02, box=0.3, lam_lo=1.0, lam_hi=20.0)
    P = gpu_problem(ctx, inst, D.FP32)
    ctx.serve_start(slots=8, hbm_budget_bytes=1 << 30)
    try:
        t = ctx.submit(P, D.opts("DFGM", eps_out=1e-3))
        st, xl, xa, lm, r = _wait(ctx, t, 10, 5)
    finally:
        ctx.serve_stop()
    xs, _, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    qp = oracle_qp(inst)
    x = xl if r.converged_last else xa
    assert O.infeas(qp, x) <= 1.01e-3 and O.F(qp, x) - fs <= 1e-3
    ctx.close()


def test_admission_rejects_what_never_fits():
    from paper_1504_05708_gb300 import duquad as D
    ctx = D.Context(0)
    big = W.single_dense(n=600, p=10, seed=1)
    small = W.single_dense(n=20, p=10, seed=2)
    Pb = gpu_problem(ctx, big, D.FP32)
    Ps = gpu_problem(ctx, small, D.FP32)
    ctx.serve_start(slots=4, hbm_budget_bytes=64 << 10)
    try:
        with pytest.raises(D.DuquadError) as e:
            ctx.submit(Pb, D.opts("DFGM"))
        assert e.value.status == D.ERR_REJECTED
        t = ctx.submit(Ps, D.opts("DFGM"))
        st, *_ = _wait(ctx, t, 20, 10)
        assert st in (0, 1)
        with pytest.raises(D.DuquadError) as e:
            ctx.poll(987654321, 20, 10)
        assert e.value.status == D.ERR_INVALID
    finally:
        ctx.serve_stop()
    ctx.close()
