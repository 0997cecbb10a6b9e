"""Sparse (CSR) problems on the grid engine (dq_problem_create_sparse), through the C ABI.

The method is unchanged for sparse Q and G (Sec. 5: only the matrix-vector products change,
to O(nnz)), so the oracle runs the same QP on the dense expansion: FP64 iterates equal the
oracle's at equal counts and in certificate mode (1e-9), FP32 solves are eps-optimal when
re-scored in FP64; at full size (n = 2e6) the first FOM steps are checked against the oracle's
FOM step with scipy.sparse products, and a certified solve is re-scored in FP64.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import ALG_IDS, rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


def _problem(ctx, d, prec, **kw):
    from paper_1504_05708_gb300 import duquad as D
    return D.SparseProblem(ctx, (d["Q_rowptr"], d["Q_col"], d["Q_val"]), d["q"],
                           (d["G_rowptr"], d["G_col"], d["G_val"]) if d["p"] else (None, None, None),
                           d["g"] if d["p"] else None, d["lb"], d["ub"], prec=prec, lmin_Q=d["lmin_Q"], **kw)


def _qp(d, cone=O.CONE_INEQ):
    return O.QP(d["Q"], d["q"], d["G"], d["g"], d["lb"], d["ub"], cone)


def _small(n=301, p=117, seed=3, g_shift=None):
    d = W.sparse_qp(n=n, p=p, deg=8, row_nnz=8, seed=seed, dense=True)
    if g_shift is not None:  # tighter constraints: some active at the optimum
        d["g"] = d["g"] * 0.02 + g_shift
    return d


@pytest.mark.parametrize("alg", ["DGM", "DFGM", "ADGM", "ADFGM"])
def test_fp64_fixed_counts_parity(ctx, alg):
    from paper_1504_05708_gb300 import duquad as D
    d = _small(g_shift=-0.05)
    qp = _qp(d)
    c = O.constants(qp, ALG_IDS[alg], lmin_Q=d["lmin_Q"])
    ro = O.dfom(qp, ALG_IDS[alg], c, inner_fixed=9, outer_fixed=5)
    P = _problem(ctx, d, D.FP64)
    xl, xa, lam, (r,) = P.solve(D.opts(alg, rho=c.rho, LL=c.LL, Ld=c.Ld, sigma=c.sigma, fixed_inner=9,
                                       fixed_outer=5))
    assert r.inner_iters == ro.inner_iters
    assert rel(xl, ro.x_last) <= 1e-9 and rel(xa, ro.x_avg) <= 1e-9
    assert rel(lam, ro.lam) <= 1e-9 or np.linalg.norm(ro.lam) == 0
    assert abs(r.f_last - ro.f_last) <= 1e-9 * max(1.0, abs(ro.f_last))


@pytest.mark.parametrize("alg", ["DFGM", "ADFGM"])
def test_fp64_certificate_mode_parity(ctx, alg):
    from paper_1504_05708_gb300 import duquad as D
    d = _small(n=240, p=90, seed=5, g_shift=-0.05)
    qp = _qp(d)
    c = O.constants(qp, ALG_IDS[alg], lmin_Q=d["lmin_Q"])
    ro = O.dfom(qp, ALG_IDS[alg], c, eps_in=1e-8, eps_out=1e-4, inner_check_every=3, outer_check_every=2,
                max_outer=5000)
    P = _problem(ctx, d, D.FP64)
    xl, xa, lam, (r,) = P.solve(D.opts(alg, rho=c.rho, LL=c.LL, Ld=c.Ld, sigma=c.sigma, eps_in=1e-8, eps_out=1e-4,
                                       inner_check_every=3, check_every=2, max_outer=5000))
    assert r.status == ro.status == 0
    assert (r.outer_iters, r.inner_iters) == (ro.outer_iters, ro.inner_iters)
    assert rel(xl, ro.x_last) <= 1e-9


def test_equality_cone_parity(ctx):
    """K = {0}, rho > 0: the sparse path keeps the two-matrix augmented form (no dense Q + rho G'G)."""
    from paper_1504_05708_gb300 import duquad as D
    d = _small(n=200, p=40, seed=8)
    u0 = np.random.default_rng(1).uniform(-0.5, 0.5, 200)
    d["g"] = -(d["G"] @ u0)
    qp = _qp(d, O.CONE_EQ)
    c = O.constants(qp, O.ADFGM, lmin_Q=d["lmin_Q"])
    ro = O.dfom(qp, O.ADFGM, c, inner_fixed=8, outer_fixed=6)
    P = _problem(ctx, d, D.FP64, cone=D.CONE_EQ)
    xl, xa, lam, (r,) = P.solve(D.opts("ADFGM", rho=c.rho, LL=c.LL, Ld=c.Ld, sigma=c.sigma, fixed_inner=8,
                                       fixed_outer=6))
    assert rel(xl, ro.x_last) <= 1e-9 and rel(lam, ro.lam) <= 1e-9


@pytest.mark.parametrize("alg", ["DFGM", "ADFGM"])
def test_fp32_eps_optimal(ctx, alg):
    from paper_1504_05708_gb300 import duquad as D
    d = W.sparse_qp(n=900, p=360, seed=9, dense=True)
    d["g"] = d["g"] * 0.02 - 0.05
    qp = _qp(d)
    eps = 1e-3
    P = _problem(ctx, d, D.FP32)
    xl, xa, lam, (r,) = P.solve(D.opts(alg, eps_out=eps, max_outer=20000))
    assert r.status == 0
    lmax, _, nG2 = P.constants()
    ev = np.linalg.eigvalsh(d["Q"])[-1]
    assert ev <= lmax <= 1.02 * ev and np.linalg.norm(d["G"], 2) ** 2 <= nG2
    ref = O.dfom(qp, O.ADFGM, O.constants(qp, O.ADFGM, lmin_Q=1.0), eps_out=1e-5, eps_in=1e-9,
                 outer_check_every=5, max_outer=5000)
    x = xl if r.converged_last else xa
    assert O.infeas(qp, x) <= eps * 1.01
    assert O.F(qp, x) - ref.d_lb <= eps * 1.01
    assert rel(x, ref.x_last) <= 1e-2


def test_bound_mode_and_device_arrays(ctx):
    import torch
    from paper_1504_05708_gb300 import duquad as D
    d = _small(n=120, p=50, seed=2)
    P = _problem(ctx, d, D.FP64, lipschitz=D.LIP_BOUND)
    lmax, _, nG2 = P.constants()
    Q, G = d["Q"], d["G"]
    assert lmax == pytest.approx(min(np.abs(Q).sum(1).max(), np.linalg.norm(Q, "fro")), rel=1e-12)
    assert nG2 == pytest.approx(min(np.abs(G).sum(0).max() * np.abs(G).sum(1).max(), np.linalg.norm(G, "fro") ** 2),
                                rel=1e-12)
    o = D.opts("DFGM", fixed_inner=5, fixed_outer=4, LL=100.0, Ld=2.0, sigma=1.0)
    xh, _, _, _ = P.solve(o)
    t = {k: torch.tensor(d[k], device="cuda") for k in ("Q_rowptr", "Q_col", "G_rowptr", "G_col")}
    v = {k: torch.tensor(d[k], dtype=torch.float64, device="cuda") for k in ("Q_val", "G_val", "q", "g", "lb", "ub")}
    Pd = D.SparseProblem(ctx, (t["Q_rowptr"], t["Q_col"], v["Q_val"]), v["q"], (t["G_rowptr"], t["G_col"], v["G_val"]),
                         v["g"], v["lb"], v["ub"], prec=D.FP64, lmin_Q=1.0)
    xd, _, _, _ = Pd.solve(o)
    assert np.array_equal(xh, xd)


def test_invalid_sparse_inputs_rejected(ctx):
    from paper_1504_05708_gb300 import duquad as D
    base = _small(n=50, p=20, seed=4)

    def bad(**mod):
        d = {k: (v.copy() if hasattr(v, "copy") else v) for k, v in base.items()}
        for k, f in mod.items():
            f(d[k])
        with pytest.raises(D.DuquadError) as e:
            _problem(ctx, d, D.FP64)
        assert e.value.status == D.ERR_INVALID
        return str(e.value)

    def asym(v):
        v[1] += 1e-3  # entry 1 of row 0 is off the diagonal: its mirror keeps the old value
    assert "symmetric" in bad(Q_val=asym)
    assert "increasing" in bad(Q_col=lambda c: c.__setitem__(slice(0, 2), c[0:2][::-1].copy()))
    assert "range" in bad(G_col=lambda c: c.__setitem__(3, 50))
    bad(G_val=lambda v: v.__setitem__(0, np.nan))
    bad(lb=lambda v: v.__setitem__(4, 2.0))
    with pytest.raises(D.DuquadError):  # sparse problems run on the grid engine only
        _problem(ctx, base, D.FP64).solve(D.opts("DFGM", engine=D.ENGINE_CTA))


def test_full_size_first_steps_and_rescored_solve(ctx):
    """n = 2e6, p = 1e6 (the sparse benchmark's size): two FOM steps of ADFGM from x^0 = 0 against
    the oracle's FOM step with scipy.sparse products, then a certified FP32 solve re-scored in FP64."""
    import scipy.sparse as sp
    import torch
    from paper_1504_05708_gb300 import duquad as D
    n, p = 2_000_000, 1_000_000
    d = W.sparse_qp(n=n, p=p, seed=6)
    Q = sp.csr_matrix((d["Q_val"], d["Q_col"], d["Q_rowptr"]), shape=(n, n))
    G = sp.csr_matrix((d["G_val"], d["G_col"], d["G_rowptr"]), shape=(p, n))
    P = _problem(ctx, d, D.FP32)
    rho, LL, sigma, Ld = 0.3, 40.0, 1.0, 2.5
    xa = torch.zeros(n, device="cuda")
    (r,) = P.solve(D.opts("ADFGM", rho=rho, LL=LL, sigma=sigma, Ld=Ld, fixed_inner=2, fixed_outer=1,
                          output=D.OUT_AVERAGE), device_out=(None, xa, None))
    torch.cuda.synchronize()
    x2 = xa.double().cpu().numpy()
    q, g, lb, ub = d["q"], d["g"], d["lb"], d["ub"]
    # the FOM step in FP32-rounded data (the problem holds FP32 values)
    Q32 = sp.csr_matrix((d["Q_val"].astype(np.float32).astype(np.float64), d["Q_col"], d["Q_rowptr"]), shape=(n, n))
    G32 = sp.csr_matrix((d["G_val"].astype(np.float32).astype(np.float64), d["G_col"], d["G_rowptr"]), shape=(p, n))
    q32, g32 = q.astype(np.float32).astype(np.float64), g.astype(np.float32).astype(np.float64)
    x1 = O.sampled_fom_step(q=q32, g=g32, G=G32, Q_rows=None, rows=None, y=np.zeros(n), mu=np.zeros(p), rho=rho,
                            L=LL, lb=lb, ub=ub, Qy_full=np.zeros(n))
    beta = (np.sqrt(LL) - np.sqrt(sigma)) / (np.sqrt(LL) + np.sqrt(sigma))
    y2 = x1 + beta * x1
    ref = O.sampled_fom_step(q=q32, g=g32, G=G32, Q_rows=None, rows=None, y=y2, mu=np.zeros(p), rho=rho, L=LL,
                             lb=lb, ub=ub, Qy_full=Q32 @ y2)
    assert np.abs(x2 - ref).max() <= 2e-5
    # certified solve, re-scored in FP64
    eps = 1e-3
    xl_t, xa_t = torch.empty(n, device="cuda"), torch.empty(n, device="cuda")
    lam_t = torch.empty(p, device="cuda")
    (r,) = P.solve(D.opts("ADFGM", eps_out=eps, eps_in=1e-5, check_every=10, inner_check_every=5,
                          max_outer=20000), device_out=(xl_t, xa_t, lam_t))
    torch.cuda.synchronize()
    assert r.status == 0
    for x_t, conv, f_dev, i_dev in ((xl_t, r.converged_last, r.f_last, r.infeas_last),
                                    (xa_t, r.converged_avg, r.f_avg, r.infeas_avg)):
        x = x_t.double().cpu().numpy()
        f64 = 0.5 * x @ (Q32 @ x) + q32 @ x
        inf64 = np.linalg.norm(np.maximum(G32 @ x + g32, 0.0))
        assert abs(f64 - f_dev) <= 1e-6 * max(1.0, abs(f64)), (f64, f_dev)
        assert abs(inf64 - i_dev) <= 1e-6, (inf64, i_dev)
        if conv:
            assert inf64 <= eps * 1.01 and f64 - r.d_lb <= eps * 1.01
