"""GPU parity of the grid engine (one large instance over the whole GPU) against the oracle."""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import ALG_IDS, exact_constants, gpu_opts_from, gpu_problem, oracle_qp, rel

pytestmark = pytest.mark.gpu
ALGS = ("DGM", "DFGM", "ADGM", "ADFGM")


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("n,p", [(301, 150), (1030, 517)])
def test_fp64_fixed_counts_parity(ctx, alg, n, p):
    """Sizes that span many row tiles with ragged tails (n, p not multiples of the vector width)."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=n, p=p, seed=7 + n, g_scale=0.05, lam_lo=1.0, lam_hi=30.0)
    c = exact_constants(inst, alg)
    ro = O.dfom(oracle_qp(inst), ALG_IDS[alg], c, inner_fixed=6, outer_fixed=4)
    P = gpu_problem(ctx, inst, D.FP64)
    xl, xa, lam, (r,) = P.solve(gpu_opts_from(c, alg, fixed_inner=6, fixed_outer=4, engine=D.ENGINE_GRID))
    assert r.inner_iters == ro.inner_iters
    assert rel(xl, ro.x_last) <= 1e-9 and rel(xa, ro.x_avg) <= 1e-9
    assert rel(lam, ro.lam) <= 1e-9 or np.linalg.norm(ro.lam) == 0


@pytest.mark.parametrize("alg", ["DFGM", "ADFGM"])
def test_fp64_certificate_mode_matches_counts(ctx, alg):
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=120, p=60, seed=3, g_scale=0.02, lam_lo=1.0, lam_hi=30.0)
    c = exact_constants(inst, alg)
    eps_in = 1e-8
    ro = O.dfom(oracle_qp(inst), ALG_IDS[alg], c, eps_in=eps_in, eps_out=1e-4, inner_check_every=3,
                outer_check_every=2, max_outer=5000)
    P = gpu_problem(ctx, inst, D.FP64)
    xl, xa, lam, (r,) = P.solve(gpu_opts_from(c, alg, eps_in=eps_in, eps_out=1e-4, inner_check_every=3,
                                                check_every=2, max_outer=5000, engine=D.ENGINE_GRID))
    assert r.status == ro.status == 0
    assert (r.outer_iters, r.inner_iters) == (ro.outer_iters, ro.inner_iters)
    assert rel(xl, ro.x_last) <= 1e-9


@pytest.mark.parametrize("alg", ["ADFGM", "ADGM"])
def test_fp32_large_dense_eps_optimal(ctx, alg):
    """The large dense generator at n = 400: FP32 solve re-scored in FP64 by the oracle."""
    from paper_1504_05708_gb300 import duquad as D
    d = W.large_dense(n=400, p=200, seed=1, device="cpu")
    import torch
    arr = {k: v.double().numpy() for k, v in d.items() if k != "lmin_Q"}
    inst = W.Instance(arr["Q"], arr["q"], arr["G"], arr["g"], arr["lb"], arr["ub"], d["lmin_Q"])
    eps = 1e-3
    P = gpu_problem(ctx, inst, D.FP32)
    xl, xa, lam, (r,) = P.solve(D.opts(alg, eps_out=eps, eps_in=1e-6, check_every=5, engine=D.ENGINE_GRID))
    assert r.status == 0
    qp = oracle_qp(inst)
    c = exact_constants(inst, alg)
    # FP64 reference run; its d_lb is a lower bound of F* whether or not it converged
    ro = O.dfom(qp, O.ADFGM, exact_constants(inst, "ADFGM"), eps_out=1e-6, eps_in=1e-9, outer_check_every=5,
                max_outer=1000)
    fstar_lb = ro.d_lb
    x = xl if r.converged_last else xa
    assert O.infeas(qp, x) <= eps * 1.01
    assert O.F(qp, x) - fstar_lb <= eps * 1.01
    assert rel(x, ro.x_last) <= 1e-2


def test_full_size_sampled_step(ctx):
    """n = 20000, p = 10000 (the large FP32 case), the launch configuration the benchmark times:
    one outer iteration of two inner FGM_sigma steps of ADFGM from x^0 = 0, checked on sampled
    coordinates against the oracle's FOM step written out in FP64 (eq. auglag1 gradient)."""
    import torch
    from paper_1504_05708_gb300 import duquad as D
    n, p = 20000, 10000
    d = W.large_dense(n=n, p=p, seed=1, device="cuda")
    rho, LL, sigma, Ld = 0.3, 6.0, 0.01, 2.5
    P = D.Problem(ctx, d["Q"], d["q"], d["G"], d["g"], d["lb"], d["ub"], prec=D.FP32, lmin_Q=0.01,
                  lmax_Q=5.0, normG2=3.0)
    xa = torch.zeros(n, device="cuda")
    o = D.opts("ADFGM", rho=rho, LL=LL, sigma=sigma, Ld=Ld, fixed_inner=2, fixed_outer=1,
               output=D.OUT_AVERAGE, engine=D.ENGINE_GRID)
    (r,) = P.solve(o, device_out=(None, xa, None))
    torch.cuda.synchronize()
    x2 = xa.double().cpu().numpy()
    rng = np.random.default_rng(0)
    idx = np.sort(rng.choice(n, 256, replace=False))
    Qs = d["Q"][torch.as_tensor(idx, device="cuda")].double().cpu().numpy()
    G = d["G"].double().cpu().numpy()
    q, g = d["q"].double().cpu().numpy(), d["g"].double().cpu().numpy()
    # x^1 = [0 - grad(0)/L]_U ; grad(0) = q + G' [rho g]_+ (= q since g < 0)
    x1 = O.sampled_fom_step(q=q, g=g, G=G, Q_rows=None, rows=None, y=np.zeros(n), mu=np.zeros(p), rho=rho,
                            L=LL, lb=-np.ones(n), ub=np.ones(n), Qy_full=np.zeros(n))
    beta = (np.sqrt(LL) - np.sqrt(sigma)) / (np.sqrt(LL) + np.sqrt(sigma))
    y2 = x1 + beta * x1
    # Q y2 at the sampled rows only
    ref = O.sampled_fom_step(q=q, g=g, G=G, Q_rows=Qs, rows=idx, y=y2, mu=np.zeros(p), rho=rho, L=LL,
                             lb=-np.ones(n), ub=np.ones(n))
    err = np.abs(x2[idx] - ref)
    assert err.max() <= 2e-5, err.max()


@pytest.mark.parametrize("alg", ["DFGM", "ADFGM"])
def test_single_pass_matches_two_pass(ctx, alg, monkeypatch):
    """FP32: the single-pass iteration (packed upper triangle of Q, one read of G) and the
    two-pass form give the same iterates at equal counts up to FP32 rounding, and both stay
    within FP32 accuracy of the FP64 oracle (sizes with ragged CTA row ranges)."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=1028, p=517, seed=41, g_scale=0.05, lam_lo=1.0, lam_hi=30.0)
    c = exact_constants(inst, alg)
    o = gpu_opts_from(c, alg, fixed_inner=7, fixed_outer=3, engine=D.ENGINE_GRID)
    P = gpu_problem(ctx, inst, D.FP32)
    monkeypatch.setenv("DQ_GRID_SINGLE_PASS", "0")
    x1, a1, l1, _ = P.solve(o)
    monkeypatch.setenv("DQ_GRID_SINGLE_PASS", "1")
    x2, a2, l2, _ = P.solve(o)
    ro = O.dfom(oracle_qp(inst), ALG_IDS[alg], c, inner_fixed=7, outer_fixed=3)
    assert rel(x2, x1) <= 2e-5 and rel(a2, a1) <= 2e-5
    assert rel(x2, ro.x_last) <= 1e-4 and rel(x1, ro.x_last) <= 1e-4


def _eq_qp(inst):
    return O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, cone=O.CONE_EQ)


def _eq_constants(inst, alg):
    return O.constants(_eq_qp(inst), ALG_IDS[alg], lmin_Q=inst.lmin_Q)


@pytest.mark.parametrize("alg", ["ADGM", "ADFGM"])
@pytest.mark.parametrize("n,p", [(301, 120), (1030, 333)])
def test_fp64_equality_hessian_mode_parity(ctx, alg, n, p):
    """K = {0}, rho > 0: the grid engine precomputes H = Q + rho G'G and runs one product
    per inner iteration; at equal counts it follows the oracle's two-matrix form to 1e-9."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.equality_dense(n=n, p=p, seed=11 + n, lam_lo=1.0, lam_hi=30.0)
    c = _eq_constants(inst, alg)
    ro = O.dfom(_eq_qp(inst), ALG_IDS[alg], c, inner_fixed=6, outer_fixed=4)
    P = gpu_problem(ctx, inst, D.FP64, cone=D.CONE_EQ)
    xl, xa, lam, (r,) = P.solve(gpu_opts_from(c, alg, fixed_inner=6, fixed_outer=4, engine=D.ENGINE_GRID))
    assert r.inner_iters == ro.inner_iters
    assert rel(xl, ro.x_last) <= 1e-9 and rel(xa, ro.x_avg) <= 1e-9
    assert rel(lam, ro.lam) <= 1e-9


def test_fp32_equality_hessian_matches_two_matrix_form(ctx, monkeypatch):
    """The Hessian mode and the two-matrix augmented form give the same FP32 iterates up to
    rounding, on a size with ragged row tiles; both stay within FP32 accuracy of the oracle."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.equality_dense(n=1028, p=301, seed=5, lam_lo=1.0, lam_hi=30.0)
    c = _eq_constants(inst, "ADFGM")
    o = gpu_opts_from(c, "ADFGM", fixed_inner=8, fixed_outer=3, engine=D.ENGINE_GRID)
    P = gpu_problem(ctx, inst, D.FP32, cone=D.CONE_EQ)
    monkeypatch.setenv("DQ_GRID_HESSIAN", "0")
    x1, a1, l1, _ = P.solve(o)
    monkeypatch.setenv("DQ_GRID_HESSIAN", "1")
    x2, a2, l2, _ = P.solve(o)
    ro = O.dfom(_eq_qp(inst), O.ADFGM, c, inner_fixed=8, outer_fixed=3)
    assert rel(x2, x1) <= 1e-4 and rel(l2, l1) <= 1e-3
    assert rel(x2, ro.x_last) <= 1e-4 and rel(x1, ro.x_last) <= 1e-4


@pytest.mark.parametrize("n,p,n_zero", [(300, 80, 0), (120, 30, 20)])
def test_fp32_equality_eps_optimal(ctx, n, p, n_zero):
    """K = {0}, Q >= 0 (singular when n_zero > 0, the paper's equality-constrained case):
    the FP32 certified output is eps-optimal when re-scored in FP64 by the oracle (its d_lb is
    a lower bound of F* whether or not its own run converged)."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.equality_dense(n=n, p=p, seed=9 + n_zero, lam_lo=1.0, lam_hi=20.0, n_zero=n_zero)
    qp = _eq_qp(inst)
    eps = 1e-3
    c = O.constants(qp, O.ADFGM, lmin_Q=inst.lmin_Q)
    ref = O.dfom(qp, O.ADFGM, c, eps_out=1e-5, eps_in=1e-6, outer_check_every=5, max_outer=3000)
    P = gpu_problem(ctx, inst, D.FP32, cone=D.CONE_EQ)
    xl, xa, lam, (r,) = P.solve(D.opts("ADFGM", eps_out=eps, eps_in=1e-5, max_outer=20000, check_every=5,
                                       engine=D.ENGINE_GRID))
    assert r.status == 0
    x = xl if r.converged_last else xa
    assert O.infeas(qp, x) <= eps * 1.01
    assert O.F(qp, x) - ref.d_lb <= eps * 1.01


@pytest.mark.parametrize("alg", ["DFGM", "ADFGM"])
def test_fp32_step_certificate(ctx, alg):
    """Single-pass FP32 inner loops stop on the step certificate (sigma > 0): a first inner
    solve stops within one iteration of the FP64 oracle stopping on the same certificate,
    and a full certificate-mode run re-scored in FP64 is eps-optimal, as is the run that
    stops on the certificate at x^k (DQ_CERT_POINT)."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=256, p=128, seed=41, g_scale=0.05, lam_lo=1.0, lam_hi=30.0)
    c = exact_constants(inst, alg)
    P = gpu_problem(ctx, inst, D.FP32)
    qp = oracle_qp(inst)
    for eps_in in (1e-3, 1e-5):
        o = gpu_opts_from(c, alg, eps_in=eps_in, fixed_outer=1, output=D.OUT_AVERAGE, engine=D.ENGINE_GRID)
        _, _, _, (r,) = P.solve(o)
        ro = O.dfom(qp, ALG_IDS[alg], c, eps_in=eps_in, outer_fixed=1, want_last=False, inner_cert_step=True)
        assert abs(r.inner_iters - ro.inner_iters) <= 1, (r.inner_iters, ro.inner_iters)
    eps = 1e-3
    ref = O.dfom(qp, ALG_IDS[alg], c, eps_out=1e-6, eps_in=1e-10, outer_check_every=5, max_outer=20000)
    runs = {}
    for cert in (D.CERT_STEP, D.CERT_POINT):
        o = gpu_opts_from(c, alg, eps_out=eps, eps_in=1e-5, check_every=5, engine=D.ENGINE_GRID, inner_cert=cert)
        xl, xa, lam, (r,) = P.solve(o)
        assert r.status == 0
        x = xl if r.converged_last else xa
        assert O.infeas(qp, x) <= eps * 1.01
        assert O.F(qp, x) - ref.d_lb <= eps * 1.01
        runs[cert] = r.inner_iters
    assert runs[D.CERT_STEP] <= 1.25 * runs[D.CERT_POINT], runs
