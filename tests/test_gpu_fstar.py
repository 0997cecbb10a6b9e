"""The paper's stop on |F(u) - F*| <= eps and dist_K(Gu + g) <= eps for a known F* (Sec. 6,
dq_solve_opts.stop_fstar), through the C ABI: FP64 iteration counts and iterates equal to the
oracle's run with the same criterion and constants, on both engines."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import ALG_IDS, exact_constants, gpu_opts_from, gpu_problem, oracle_qp, rel

pytestmark = pytest.mark.gpu
EPS = 1e-2


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


def _fstar(inst):
    qp = oracle_qp(inst)
    r = O.dfom(qp, O.ADFGM, exact_constants(inst, "ADFGM"), eps_out=1e-7, eps_in=1e-11, outer_check_every=5,
               max_outer=50000)
    return O.F(qp, r.x_last if r.converged_last else r.x_avg)


@pytest.mark.parametrize("want", ["last", "average"])
@pytest.mark.parametrize("alg", ["DGM", "DFGM", "ADGM", "ADFGM"])
@pytest.mark.parametrize("engine_name,n,p", [("CTA", 50, 25), ("GRID", 301, 150)])
def test_fstar_stop_matches_oracle(ctx, engine_name, n, p, alg, want):
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=n, p=p, seed=3 + n, g_scale=0.02, lam_lo=1.0, lam_hi=30.0)
    fs = _fstar(inst)
    c = exact_constants(inst, alg)
    eps_in = O.default_eps_in(ALG_IDS[alg], EPS, c.Ld)
    ro = O.dfom(oracle_qp(inst), ALG_IDS[alg], c, eps_out=EPS, eps_in=eps_in, max_outer=100000, f_star=fs,
                want_last=want == "last", want_avg=want == "average")
    P = gpu_problem(ctx, inst, D.FP64)
    xl, xa, lam, (r,) = P.solve(gpu_opts_from(c, alg, eps_out=EPS, eps_in=eps_in, max_outer=100000, f_star=fs,
                                                output=D.OUT_LAST if want == "last" else D.OUT_AVERAGE,
                                                engine=getattr(D, "ENGINE_" + engine_name)))
    assert r.status == ro.status == 0
    assert (r.outer_iters, r.inner_iters) == (ro.outer_iters, ro.inner_iters)
    x, xo = (xl, ro.x_last) if want == "last" else (xa, ro.x_avg)
    assert rel(x, xo) <= 1e-9
    qp = oracle_qp(inst)
    assert abs(O.F(qp, x) - fs) <= EPS and O.infeas(qp, x) <= EPS
