"""Theory mode on the GPU (dq_solve_theory), through the C ABI.

With eps_in and k_out of eq. choose_ein, the FOM count k_in of Sec. 5 and lambda^0 = 0, the
averaged primal output of the GPU solve satisfies the theorems' bounds, checked in FP64 by the
oracle against brute-force KKT: (A)DGM dist_K <= eps / R_d and -eps <= F - F* <= eps / 4;
(A)DFGM dist_K <= 3 eps / R_d and -3 eps <= F - F* <= 5 eps / 4 (ADGM/ADFGM at
rho* = 8 R_d^2 / eps).  R_d is either the exact ||lambda*|| or the library's estimate (safety
times the norm of a certified solve's multipliers), which must not fall below ||lambda*||.
"""
import math

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import ALG_IDS, gpu_problem, oracle_qp

pytestmark = pytest.mark.gpu
EPS = 1e-2


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


def _instances(count=3):
    from oracle.kkt import solve_kkt
    out = []
    for seed in range(1, 40):
        inst = W.single_dense(n=5, p=4, seed=seed, lam_lo=1.0, lam_hi=10.0, g_scale=0.02, box=0.3)
        xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
        if np.linalg.norm(lam_s) >= 0.1:  # some constraint active: something to certify
            out.append((inst, float(np.linalg.norm(lam_s)), fs))
        if len(out) == count:
            return out
    raise AssertionError("too few instances with active constraints")


@pytest.mark.parametrize("estimate", [False, True])
@pytest.mark.parametrize("alg", ["DGM", "DFGM", "ADGM", "ADFGM"])
def test_theory_counts_meet_the_primal_bounds_on_gpu(ctx, alg, estimate):
    from paper_1504_05708_gb300 import duquad as D
    fast = alg in ("DFGM", "ADFGM")
    for inst, Rd, fs in _instances():
        P = gpu_problem(ctx, inst, D.FP64, lmax_Q=float(np.linalg.eigvalsh(inst.Q)[-1]),
                        normG2=float(np.linalg.norm(inst.G, 2) ** 2))
        xl, xa, lam, r, counts, rd_used = P.solve_theory(alg, EPS, Rd=math.nan if estimate else Rd,
                                                         engine=D.ENGINE_CTA, max_total=200_000_000)
        assert r.status == 0 and r.outer_iters == counts["k_out"]
        assert r.inner_iters >= counts["k_out"] * counts["k_in"]
        if estimate:
            assert rd_used >= Rd, (rd_used, Rd)
        else:
            assert rd_used == Rd
        # the counts are dq_theory's for this R_d
        qp = oracle_qp(inst)
        a = ALG_IDS[alg]
        rho = O.rho_star(EPS, rd_used) if a in (O.ADGM, O.ADFGM) else 0.0
        c = O.constants(qp, a, rho=rho, lmin_Q=inst.lmin_Q)
        assert counts["k_out"] == max(1, math.ceil(O.k_out(a, EPS, c.Ld, rd_used) * (1 - 1e-14)))
        assert r.rho == pytest.approx(rho, rel=1e-15)
        # the theorems' primal bounds on the averaged output, re-scored in FP64 against F*
        inf, f = O.infeas(qp, xa), O.F(qp, xa)
        assert inf <= (3.0 if fast else 1.0) * EPS / Rd, (inf, Rd)
        assert -(3.0 if fast else 1.0) * EPS <= f - fs <= (1.25 if fast else 0.25) * EPS, (f - fs)
        # and the same run by the oracle with the same counts agrees to FP64 rounding
        ro = O.dfom(qp, a, c, inner_fixed=counts["k_in"], outer_fixed=counts["k_out"],
                    eps_in=counts["eps_in"])
        assert np.linalg.norm(xa - ro.x_avg) <= 1e-9 * max(1.0, np.linalg.norm(ro.x_avg))
        P.close()


def test_theory_cap_refuses_before_solving(ctx):
    from paper_1504_05708_gb300 import duquad as D
    inst, Rd, _ = _instances(1)[0]
    P = gpu_problem(ctx, inst, D.FP64)
    with pytest.raises(D.DuquadError) as e:
        P.solve_theory("DGM", 1e-6, Rd=Rd, max_total=1000)
    assert e.value.status == D.ERR_INVALID and "exceeds the cap" in str(e.value)
