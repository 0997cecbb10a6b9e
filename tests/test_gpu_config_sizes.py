"""Oracle re-scoring at the workloads' own sizes, through the C ABI.

* Uneven persistent launch: one dq_solve_many launch over FP32 instances drawn like the uneven
  batch at n in {160, 256, 384, 512} (past the size where the thread-block engine stops staging
  Q in shared memory), kappa(Q) up to 1e4, all four algorithms.  Each result is re-scored in
  FP64 by the oracle (infeasibility, F - a certified lower bound on F*) and compared with the
  oracle's run of the same algorithm with the same constants.
* Large dense case at full size (n = 20000, p = 10000), the launch configuration the benchmark
  times: one certified FP32 ADFGM solve, re-scored in FP64 by the oracle at full size (F, the
  infeasibility, and L_rho(x, lambda) - cert(x, lambda) as a lower bound of F*: the inner
  certificate bounds L_rho(x, lambda) - d_rho(lambda) and d_rho(lambda) <= F*).
* Shared-matrix MPC batch on tensor cores: every instance re-scored, and whichever output the
  solve returns compared with the oracle's output of the same kind.
"""
from concurrent.futures import ThreadPoolExecutor

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import ALG_IDS, exact_constants, gpu_opts_from, gpu_problem, oracle_qp, rel

pytestmark = pytest.mark.gpu
EPS = 1e-3


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


def _pool(fn, items):
    # the oracle is C called through ctypes, which releases the GIL: threads run it in parallel
    with ThreadPoolExecutor(max_workers=16) as ex:
        return list(ex.map(fn, items))


def test_uneven_persistent_launch_vs_oracle(ctx):
    from paper_1504_05708_gb300 import duquad as D
    ns = (160, 256, 384, 512)
    kappas = np.geomspace(10.0, 1e4, 10)
    insts = []
    for i in range(40):
        n, alg, kap = ns[i % 4], (i // 4) % 4, float(kappas[i // 4])
        insts.append(W.uneven_instance(n, kap, alg, 1000 + i))
    cons = [exact_constants(inst, inst.alg) for inst in insts]
    eps_in = [O.default_eps_in(ALG_IDS[inst.alg], EPS, c.Ld) for inst, c in zip(insts, cons)]
    probs = [gpu_problem(ctx, inst, D.FP32) for inst in insts]
    ops = [gpu_opts_from(c, inst.alg, eps_out=EPS, eps_in=e, max_outer=50000, engine=D.ENGINE_CTA)
           for inst, c, e in zip(insts, cons, eps_in)]
    outs, res = D.solve_many(probs, ops)

    def ref(i):
        inst, c = insts[i], cons[i]
        qp = oracle_qp(inst)
        same = O.dfom(qp, ALG_IDS[inst.alg], c, eps_out=EPS, eps_in=eps_in[i], max_outer=50000)
        lower = O.dfom(qp, O.ADFGM, exact_constants(inst, "ADFGM"), eps_out=1e-6, eps_in=1e-10,
                       outer_check_every=5, max_outer=20000)
        return same, lower.d_lb

    refs = _pool(ref, range(len(insts)))
    for i, (inst, (xl, xa, _), r, (same, f_lb)) in enumerate(zip(insts, outs, res, refs)):
        qp = oracle_qp(inst)
        assert r.status == 0 and same.status == 0, (i, inst.alg, r.status, same.status)
        x, xo = (xl[0], same.x_last) if r.converged_last else (xa[0], same.x_avg)
        assert O.infeas(qp, x) <= EPS * 1.01, (i, O.infeas(qp, x))
        assert O.F(qp, x) - f_lb <= EPS * 1.01, (i, O.F(qp, x) - f_lb)
        assert rel(x, xo) <= 1e-3, (i, inst.n, inst.alg, inst.meta["kappa"], rel(x, xo))


def test_large_dense_full_size_rescored(ctx):
    import torch
    from paper_1504_05708_gb300 import duquad as D
    n, p = 20000, 10000
    d = W.large_dense(n=n, p=p, seed=1, device="cuda")
    P = D.Problem(ctx, d["Q"], d["q"], d["G"], d["g"], d["lb"], d["ub"], prec=D.FP32, lmin_Q=0.01)
    xl = torch.empty(n, device="cuda")
    xa = torch.empty(n, device="cuda")
    lam = torch.empty(p, device="cuda")
    o = D.opts("ADFGM", eps_out=EPS, eps_in=1e-5, check_every=10, inner_check_every=5, engine=D.ENGINE_GRID)
    (r,) = P.solve(o, device_out=(xl, xa, lam))
    torch.cuda.synchronize()
    assert r.status == 0 and (r.converged_last or r.converged_avg)
    qp = O.QP(*(d[k].double().cpu().numpy() for k in ("Q", "q", "G", "g", "lb", "ub")))
    del d
    x_last, x_avg, lm = (t.double().cpu().numpy() for t in (xl, xa, lam))
    rho, LL, sigma = r.rho, r.LL, r.sigma
    assert np.all(lm >= 0) and np.all(np.abs(x_last) <= 1) and np.all(np.abs(x_avg) <= 1)
    # a certified lower bound of F* from the returned pair (x_last = ubar(lambda^k), lambda^k)
    f_lb = O.lagrangian(qp, rho, x_last, lm) - O.inner_cert(qp, rho, x_last, lm, LL, sigma)
    for x, conv, f_dev, i_dev in ((x_last, r.converged_last, r.f_last, r.infeas_last),
                                  (x_avg, r.converged_avg, r.f_avg, r.infeas_avg)):
        f64, inf64 = O.F(qp, x), O.infeas(qp, x)
        assert abs(f64 - f_dev) <= 1e-6 * max(1.0, abs(f64)), (f64, f_dev)
        assert abs(inf64 - i_dev) <= 1e-6, (inf64, i_dev)
        if conv:
            assert inf64 <= EPS * 1.01, inf64
            assert f64 - f_lb <= EPS * 1.01, (f64, f_lb)
    assert f_lb <= r.d_lb + 1e-6 * max(1.0, abs(f_lb)) or f_lb <= min(O.F(qp, x_last), O.F(qp, x_avg))


@pytest.mark.parametrize("alg", ["DGM", "DFGM"])
def test_mpc_every_instance_rescored(ctx, alg):
    from paper_1504_05708_gb300 import duquad as D
    B = 130
    d = W.mpc_batch(batch=B, seed=5)
    lmin = float(np.linalg.eigvalsh(d["Q"])[0]) * 0.999
    P = D.Problem(ctx, d["Q"], d["qs"], d["G"], d["gs"], d["lb"], d["ub"], prec=D.BF16X3, batch=B, lmin_Q=lmin)
    max_outer = 200000 if alg == "DGM" else 20000
    xl, xa, lam, res = P.solve(D.opts(alg, eps_out=EPS, eps_in=1e-5, check_every=5, max_outer=max_outer))
    bad = [(b, r.status, r.outer_iters) for b, r in enumerate(res) if r.status != 0]
    assert not bad, bad[:10]
    lmax = float(np.linalg.eigvalsh(d["Q"])[-1])
    e_lmax, _, e_nG2 = P.constants()

    def ref(b):
        qp = O.QP(d["Q"], d["qs"][b], d["G"], d["gs"][b], d["lb"], d["ub"])
        # the solve's own constants, so that both sides take the same steps
        r = res[b]
        c = O.Constants(r.rho, r.LL, r.sigma, r.Ld, e_lmax, lmin, e_nG2)
        same = O.dfom(qp, ALG_IDS[alg], c, eps_in=1e-5, eps_out=EPS, outer_check_every=5, max_outer=max_outer)
        lower = O.dfom(qp, O.DFGM, O.constants(qp, O.DFGM, lmin_Q=lmin, lmax_Q=lmax), eps_in=1e-9,
                       eps_out=1e-5, outer_check_every=10, max_outer=50000)
        return same, lower.d_lb

    refs = _pool(ref, range(B))
    worst = 0.0
    for b, (same, f_lb) in enumerate(refs):
        qp = O.QP(d["Q"], d["qs"][b], d["G"], d["gs"][b], d["lb"], d["ub"])
        x, xo = (xl[b], same.x_last) if res[b].converged_last else (xa[b], same.x_avg)
        assert O.infeas(qp, x) <= EPS * 1.01, (b, O.infeas(qp, x))
        assert O.F(qp, x) - f_lb <= EPS * 1.01, (b, O.F(qp, x) - f_lb)
        worst = max(worst, rel(x, xo))
        assert rel(x, xo) <= 1e-3, (b, res[b].converged_last, res[b].outer_iters, same.outer_iters, rel(x, xo))
