"""Pins of the FP64 oracle against facts fixed by the paper and by mathematics.

None of these re-types the oracle's formulas: each compares it with a closed
form, a hand-derived worked example (tests/golden), an independent route
(brute-force KKT enumeration, scipy minimisation, finite differences, LAPACK
eigenvalues) or an exact algebraic relation the paper derives (identity_lag,
S_k = theta_k^2, the averaged-iterate feasibility identity), chosen so that a
dropped term, a wrong sign, a wrong step size or a shifted index fails one.
"""
import json
import math
import os

import numpy as np
import pytest

import oracle as O
import workloads as W
from oracle.kkt import solve_kkt

GOLD = os.path.join(os.path.dirname(__file__), "golden")
ALGS = (O.DGM, O.DFGM, O.ADGM, O.ADFGM)


def _qp(inst, cone=O.CONE_INEQ):
    return O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, cone)


def _golden(name):
    with open(os.path.join(GOLD, name)) as f:
        d = json.load(f)
    qp = O.QP(np.array(d["Q"]), np.array(d["q"]), np.array(d["G"]), np.array(d["g"]),
              np.array(d["lb"]), np.array(d["ub"]))
    return qp, d


def _small(seed, n=6, p=4, g_scale=0.02, box=1.0):
    inst = W.single_dense(n=n, p=p, seed=seed, lam_lo=1.0, lam_hi=10.0, g_scale=g_scale, box=box)
    return inst, _qp(inst)


# --------------------------------------------------------------- worked examples

@pytest.mark.parametrize("name", ["two_var_qp.json", "box_and_constraint_qp.json"])
@pytest.mark.parametrize("alg", ALGS)
def test_golden_worked_example(name, alg):
    qp, d = _golden(name)
    c = O.constants(qp, alg)
    r = O.dfom(qp, alg, c, eps_in=1e-13, eps_out=1e-9, max_outer=200000, max_inner=100000)
    assert r.status == 0
    np.testing.assert_allclose(r.x_last, d["x_star"], atol=2e-5)
    assert abs(r.f_last - d["F_star"]) < 1e-6
    # the averaged output converges at O(1/k) (DGM) / O(1/k^2) (DFGM): looser target
    ra = O.dfom(qp, alg, c, eps_in=1e-10, eps_out=1e-4, max_outer=400000, want_last=False)
    assert ra.status == 0 and ra.converged_avg
    np.testing.assert_allclose(ra.x_avg, d["x_star"], atol=1e-2)
    assert abs(ra.f_avg - d["F_star"]) < 1e-3
    if alg in (O.DGM, O.DFGM):  # rho = 0: the dual iterate is the Lagrange multiplier
        np.testing.assert_allclose(r.lam, d["lambda_star"], atol=1e-3)


def test_golden_kkt_enumeration_agrees():
    for name in ("two_var_qp.json", "box_and_constraint_qp.json"):
        qp, d = _golden(name)
        x, lam, f = solve_kkt(qp.Q, qp.q, qp.G, qp.g, qp.lb, qp.ub)
        np.testing.assert_allclose(x, d["x_star"], atol=1e-12)
        np.testing.assert_allclose(lam, d["lambda_star"], atol=1e-12)
        assert abs(f - d["F_star"]) < 1e-12


# ------------------------------------------------------------------ closed forms

@pytest.mark.parametrize("variant", [O.INNER_GM, O.INNER_FGM, O.INNER_FGMSIGMA])
def test_fom_box_only_diagonal_closed_form(variant):
    """p = 0 (Sec. 3: FOM applied directly when X_QP is simple): diagonal Q gives clamp(-q/Q_ii)."""
    rng = np.random.default_rng(5)
    n = 12
    d = rng.uniform(0.5, 5.0, n)
    q = rng.standard_normal(n) * 4
    qp = O.QP(np.diag(d), q, np.zeros((0, n)), np.zeros(0), -np.ones(n), np.ones(n))
    x, k, _ = O.fom(qp, 0.0, np.zeros(1), d.max(), d.min(), np.zeros(n), variant=variant,
                    fixed=3000)
    np.testing.assert_allclose(x, np.clip(-q / d, -1, 1), atol=1e-12)


def test_fom_unconstrained_interior():
    """Interior minimiser: FOM converges to -Q^{-1} q when the box is inactive."""
    inst = W.single_dense(n=20, p=0, seed=3, lam_lo=1.0, lam_hi=20.0, box=1e3)
    qp = _qp(inst)
    xs = -np.linalg.solve(inst.Q, inst.q)
    x, _, _ = O.fom(qp, 0.0, np.zeros(1), inst.lmax_Q, inst.lmin_Q, np.zeros(20), fixed=2000)
    np.testing.assert_allclose(x, xs, rtol=1e-10, atol=1e-10)


@pytest.mark.parametrize("alg", ALGS)
def test_single_constraint_closed_form(alg):
    """One constraint a'x + g <= 0, inactive box: lambda* = max(0, (g - a'Q^-1 q)/(a'Q^-1 a))."""
    inst = W.single_dense(n=8, p=1, seed=11, lam_lo=1.0, lam_hi=5.0, box=1e3)
    a = inst.G[0]
    Qi_q = np.linalg.solve(inst.Q, inst.q)
    Qi_a = np.linalg.solve(inst.Q, a)
    g = float(a @ Qi_q + 0.5)  # makes the unconstrained minimiser violate the constraint
    lam = max(0.0, (g - a @ Qi_q) / (a @ Qi_a))
    xs = -(Qi_q + lam * Qi_a)
    qp = O.QP(inst.Q, inst.q, a[None, :], np.array([g]), inst.lb, inst.ub)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    r = O.dfom(qp, alg, c, eps_in=1e-14, eps_out=1e-10, max_outer=200000)
    np.testing.assert_allclose(r.x_last, xs, atol=1e-5)
    if alg in (O.DGM, O.DFGM):
        assert abs(r.lam[0] - lam) < 1e-4


def test_inactive_constraints_keep_lambda_zero():
    """lambda^0 = 0 and G ubar + g < 0 at every inner solution: the update of Algorithm DFOM keeps lambda = 0."""
    inst = W.single_dense(seed=0)  # the n=50, p=25 FP64 case: constraints inactive
    qp = _qp(inst)
    for alg in (O.DGM, O.DFGM):
        c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
        r = O.dfom(qp, alg, c, inner_fixed=200, outer_fixed=5)
        assert np.all(r.lam == 0.0)


# --------------------------------------------------------------- brute force KKT

@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("alg", ALGS)
def test_matches_kkt_enumeration_box_active(seed, alg):
    inst, qp = _small(seed, n=5, p=4, g_scale=0.02, box=0.3)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    r = O.dfom(qp, alg, c, eps_in=1e-12, eps_out=1e-8, max_outer=400000)
    assert r.status == 0
    np.testing.assert_allclose(r.x_last, xs, atol=1e-3)
    assert abs(r.f_last - fs) <= 1e-7 + 1e-6 * abs(fs)
    assert r.d_lb <= fs + 1e-10          # the certificate's lower bound never exceeds F*


@pytest.mark.parametrize("seed", [4, 5])
def test_matches_kkt_enumeration_wide_box(seed):
    inst, qp = _small(seed, n=8, p=9, g_scale=0.02, box=50.0)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, box_active=False)
    for alg in ALGS:
        c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
        r = O.dfom(qp, alg, c, eps_in=1e-12, eps_out=1e-8, max_outer=400000)
        np.testing.assert_allclose(r.x_last, xs, atol=1e-4)


def test_equality_cone_matches_kkt():
    """K = {0} (equality constraints, Sec. 2): K_d = R^p."""
    inst, _ = _small(7, n=6, p=2, box=50.0)
    qp = O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, O.CONE_EQ)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, box_active=False,
                              equality=True)
    for alg in (O.DFGM, O.ADFGM):
        c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
        r = O.dfom(qp, alg, c, eps_in=1e-12, eps_out=1e-9, max_outer=400000)
        np.testing.assert_allclose(r.x_last, xs, atol=1e-5)


# --------------------------------------------- Lagrangian, gradients, definitions

@pytest.mark.parametrize("rho", [0.0, 0.7])
@pytest.mark.parametrize("cone", [O.CONE_INEQ, O.CONE_EQ])
def test_lagrangian_is_min_over_s(rho, cone):
    """eq. auglag1 equals the minimum over s in K of eq. auglag (scipy L-BFGS-B on s)."""
    from scipy.optimize import minimize
    inst, _ = _small(8, n=6, p=5, g_scale=1.0)
    qp = O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, cone)
    rng = np.random.default_rng(0)
    for _ in range(3):
        u = rng.uniform(-1, 1, 6)
        lam = rng.standard_normal(5)
        r = inst.G @ u + inst.g
        Fu = 0.5 * u @ inst.Q @ u + inst.q @ u
        if cone == O.CONE_EQ or rho == 0.0:
            # K = {0} forces s = 0; rho = 0 with K = R^p_- is linear in s and the
            # formula of eq. auglag1 takes s = 0 (the value at s(u, lambda))
            ref = Fu + lam @ r + 0.5 * rho * r @ r
        else:
            obj = lambda s: lam @ (r - s) + 0.5 * rho * (r - s) @ (r - s)
            jac = lambda s: -lam - rho * (r - s)
            m = minimize(obj, np.minimum(r, 0), jac=jac, bounds=[(None, 0.0)] * 5, method="L-BFGS-B",
                         options=dict(ftol=1e-15, gtol=1e-12))
            ref = Fu + m.fun
        assert abs(O.lagrangian(qp, rho, u, lam) - ref) < 1e-9


@pytest.mark.parametrize("rho", [0.0, 0.7])
def test_grad_lagr_finite_differences(rho):
    inst, qp = _small(9, n=7, p=5, g_scale=0.02)
    rng = np.random.default_rng(1)
    u = rng.uniform(-1, 1, 7)
    lam = np.abs(rng.standard_normal(5))
    gr = O.grad_lagr(qp, rho, u, lam)
    h = 1e-6
    fd = np.array([(O.lagrangian(qp, rho, u + h * e, lam) - O.lagrangian(qp, rho, u - h * e, lam)) / (2 * h)
                   for e in np.eye(7)])
    np.testing.assert_allclose(gr, fd, atol=1e-7)


def _dual_value(qp, rho, lam, c):
    x, _, _ = O.fom(qp, rho, lam, c.LL, c.sigma, np.zeros(qp.n), eps_in=1e-15, max_inner=20000)
    return O.lagrangian(qp, rho, x, lam), x


@pytest.mark.parametrize("alg", [O.DFGM, O.ADFGM])
def test_dual_gradient_matches_finite_differences(alg):
    """eq. Ld: grad d_rho(lambda) = G u(lambda) + g - s(u(lambda), lambda)."""
    inst, qp = _small(10, n=6, p=4, g_scale=0.02, box=0.5)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    lam = np.array([0.3, 0.0, 0.8, 0.1])
    _, x = _dual_value(qp, c.rho, lam, c)
    grad = O.dual_grad(qp, c.rho, x, lam)
    h = 1e-5
    fd = np.array([(_dual_value(qp, c.rho, lam + h * e, c)[0] - _dual_value(qp, c.rho, lam - h * e, c)[0]) / (2 * h)
                   for e in np.eye(4)])
    np.testing.assert_allclose(grad, fd, atol=2e-6)


@pytest.mark.parametrize("alg", [O.DFGM, O.ADFGM])
def test_dual_lipschitz_constant(alg):
    """L_d of eq. Ld bounds ||grad d(l1) - grad d(l2)|| / ||l1 - l2||."""
    inst, qp = _small(12, n=6, p=4, g_scale=0.02, box=0.5)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    rng = np.random.default_rng(2)
    for _ in range(5):
        l1, l2 = np.abs(rng.standard_normal(4)) * 3, np.abs(rng.standard_normal(4)) * 3
        _, x1 = _dual_value(qp, c.rho, l1, c)
        _, x2 = _dual_value(qp, c.rho, l2, c)
        g1, g2 = O.dual_grad(qp, c.rho, x1, l1), O.dual_grad(qp, c.rho, x2, l2)
        assert np.linalg.norm(g1 - g2) <= c.Ld * np.linalg.norm(l1 - l2) * (1 + 1e-9)


def test_power_iteration_matches_lapack():
    inst = W.single_dense(n=40, p=20, seed=13)
    qp = _qp(inst)
    assert abs(O.power_lmax(qp, "Q", 3000) - np.linalg.eigvalsh(inst.Q)[-1]) < 1e-8 * inst.lmax_Q
    assert abs(O.power_lmax(qp, "GtG", 3000) - np.linalg.norm(inst.G, 2) ** 2) < 1e-8


# ------------------------------------------------------ invariants of the paper

@pytest.mark.parametrize("alg", ALGS)
def test_identity_lag_every_outer(alg):
    """eq. identity_lag: dbar(mu) - <grad dbar(mu), mu> = F(ubar) + rho/2 ||grad dbar(mu)||^2."""
    inst, qp = _small(14, n=10, p=8, g_scale=0.02)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    r = O.dfom(qp, alg, c, eps_in=1e-8, outer_fixed=40, trace_cap=40)
    t = r.trace
    lhs = t[:, 5] - t[:, 6]
    rhs = t[:, 7] + 0.5 * c.rho * t[:, 8]
    np.testing.assert_allclose(lhs, rhs, atol=1e-11)
    assert np.all(t[:, 9] >= 0.0)  # lambda^k in K_d = R^p_+


@pytest.mark.parametrize("alg", [O.DFGM, O.ADFGM])
def test_theta_sequence(alg):
    """eq. fg_step: (k+1)/2 <= theta_k <= k and S_k = sum theta_j = theta_k^2."""
    inst, qp = _small(15)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    r = O.dfom(qp, alg, c, inner_fixed=5, outer_fixed=60, trace_cap=60)
    k, th, S = r.trace[:, 0], r.trace[:, 1], r.trace[:, 2]
    assert np.all((k + 1) / 2 <= th + 1e-12) and np.all(th <= k + 1e-12)
    np.testing.assert_allclose(S, th ** 2, rtol=1e-12)
    # momentum weight beta_k = (theta_k - 1)/theta_{k+1}
    np.testing.assert_allclose(r.trace[:-1, 3], (th[:-1] - 1) / th[1:], rtol=1e-12)


@pytest.mark.parametrize("alg", ALGS)
def test_box_and_dual_cone_invariants(alg):
    inst, qp = _small(16, n=12, p=10, g_scale=0.02, box=0.4)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    r = O.dfom(qp, alg, c, eps_in=1e-7, outer_fixed=30)
    assert np.all(r.x_last >= -0.4) and np.all(r.x_last <= 0.4)
    assert np.all(r.x_avg >= -0.4 - 1e-15) and np.all(r.x_avg <= 0.4 + 1e-15)
    assert np.all(r.lam >= 0.0)


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("K", [1, 2, 7, 25])
def test_average_feasibility_identity(alg, K):
    """Averaged-iterate feasibility (Sec. 4.2, proofs of eq. feasibility_final and eq. infes_av):
    with l^k = lambda^{k-1} + theta_k (lambda^k - lambda^{k-1}), summing the dual steps gives
    dist_K(G uhat^k + g) <= (2 L_d / S_k) ||l^k - lambda^0||  exactly (inexact inner solves
    included).  The paper prints the factor L_d / S_k; the summation it describes gives 2 L_d / S_k.
    DGM is the case theta = 1, S_k = k, l^k = lambda^k."""
    inst, qp = _small(17, n=10, p=8, g_scale=0.02)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    kw = dict(eps_in=1e-4, want_last=False)
    rK = O.dfom(qp, alg, c, outer_fixed=K, trace_cap=K, **kw)
    lam_prev = O.dfom(qp, alg, c, outer_fixed=K - 1, **kw).lam if K > 1 else np.zeros(qp.p)
    theta_K, S_K = rK.trace[-1, 1], rK.trace[-1, 2]
    l_K = lam_prev + theta_K * (rK.lam - lam_prev)
    bound = 2 * c.Ld / S_K * np.linalg.norm(l_K)
    assert O.infeas(qp, rK.x_avg) <= bound * (1 + 1e-10) + 1e-14


# ---------------------------------------------------------- rate bounds of the paper

@pytest.mark.parametrize("variant,power", [(O.INNER_GM, 1), (O.INNER_FGM, 2)])
def test_fom_rate_lemma(variant, power):
    """eq. bound_gen_dfg1 with sigma = 0: phi(x^k) - phi* <= 2 L R^2 / (k+1)^{p(beta)}."""
    inst, qp = _small(18, n=10, p=6, g_scale=0.02, box=0.5)
    mu = np.full(6, 0.5)
    LL = inst.lmax_Q
    xstar, _, _ = O.fom(qp, 0.0, mu, LL, inst.lmin_Q, np.zeros(10), fixed=20000)
    phistar = O.lagrangian(qp, 0.0, xstar, mu)
    R2 = float(np.sum(xstar ** 2))
    _, _, phi = O.fom(qp, 0.0, mu, LL, 0.0, np.zeros(10), variant=variant, fixed=300, phi_trace=300)
    k = np.arange(1, 301)
    assert np.all(phi - phistar <= 2 * LL * R2 / (k + 1.0) ** power + 1e-12)


def test_fom_rate_lemma_strongly_convex():
    """eq. bound_gen_dfg1 with sigma > 0 (FGM_sigma): (1 - sqrt(sigma/L))^{k-1} L R^2."""
    inst, qp = _small(19, n=10, p=6, g_scale=0.02, box=0.5)
    mu = np.full(6, 0.5)
    L, s = inst.lmax_Q, inst.lmin_Q
    xstar, _, _ = O.fom(qp, 0.0, mu, L, s, np.zeros(10), fixed=20000)
    phistar = O.lagrangian(qp, 0.0, xstar, mu)
    R2 = float(np.sum(xstar ** 2))
    _, _, phi = O.fom(qp, 0.0, mu, L, s, np.zeros(10), variant=O.INNER_FGMSIGMA, fixed=200,
                      phi_trace=200)
    k = np.arange(1, 201)
    bound = np.minimum((1 - math.sqrt(s / L)) ** (k - 1) * L * R2, 2 * L * R2 / (k + 1.0) ** 2)
    assert np.all(phi - phistar <= bound + 1e-12)


@pytest.mark.parametrize("alg,power", [(O.DGM, 1), (O.DFGM, 2), (O.ADGM, 1), (O.ADFGM, 2)])
def test_dual_rate_theorem(alg, power):
    """eq. bound_gen_dfg: F* - d_rho(lambda^k) <= 4 L_d R_d^2/(k+1)^p + 2 (k+1)^{p-1} eps_in."""
    inst, qp = _small(20, n=5, p=4, g_scale=0.02, box=0.3)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    # R_d = dist(lambda^0 = 0, Lambda*); Lambda* of the augmented dual contains lambda*
    Rd = float(np.linalg.norm(lam_s))
    eps_in = 1e-6
    for k in (1, 3, 10, 30):
        r = O.dfom(qp, alg, c, eps_in=eps_in, outer_fixed=k, want_last=False)
        d_k, _ = _dual_value(qp, c.rho, r.lam, c)
        assert fs - d_k <= 4 * c.Ld * Rd ** 2 / (k + 1) ** power + 2 * (k + 1) ** (power - 1) * eps_in + 1e-12


def test_dgm_dual_sequence_bound():
    """eq. bound_seq_dgm: ||lambda^k - lambda*|| <= R_d + sqrt(k eps_in / L_d) (DGM)."""
    inst, qp = _small(21, n=5, p=4, g_scale=0.02, box=0.3)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    c = O.constants(qp, O.DGM, lmin_Q=inst.lmin_Q)
    Rd = float(np.linalg.norm(lam_s))
    eps_in = 1e-5
    for k in (1, 5, 20, 80):
        r = O.dfom(qp, O.DGM, c, eps_in=eps_in, outer_fixed=k, want_last=False)
        assert np.linalg.norm(r.lam - lam_s) <= Rd + math.sqrt(k * eps_in / c.Ld) + 1e-12


@pytest.mark.parametrize("alg", ALGS)
def test_certificate_implies_eps_optimality(alg):
    """A converged run (certificate mode) is eps-primal optimal against brute-force F*."""
    inst, qp = _small(22, n=5, p=4, g_scale=0.02, box=0.3)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    eps = 1e-3
    r = O.dfom(qp, alg, c, eps_in=O.default_eps_in(alg, eps, c.Ld), eps_out=eps, max_outer=100000)
    assert r.status == 0
    assert r.d_lb <= fs + 1e-12
    if r.converged_last:
        assert r.infeas_last <= eps and r.f_last - fs <= eps
        assert fs - r.f_last <= np.linalg.norm(lam_s) * r.infeas_last + 1e-12
    if r.converged_avg:
        assert r.infeas_avg <= eps and r.f_avg - fs <= eps


def test_inner_fixed_count_bound_strongly_convex():
    """Sec. 5: k_in = sqrt(L/sigma) log(L D_U^2 / eps_in) + 1 iterations of FGM_sigma give an eps_in-solution."""
    inst, qp = _small(23, n=10, p=6, g_scale=0.02, box=0.5)
    mu = np.full(6, 0.3)
    L, s = inst.lmax_Q, inst.lmin_Q
    D2 = float(np.sum((inst.ub - inst.lb) ** 2))
    xstar, _, _ = O.fom(qp, 0.0, mu, L, s, np.zeros(10), fixed=20000)
    phistar = O.lagrangian(qp, 0.0, xstar, mu)
    for eps_in in (1e-3, 1e-6):
        kin = int(math.ceil(math.sqrt(L / s) * math.log(L * D2 / eps_in) + 1))
        x, _, _ = O.fom(qp, 0.0, mu, L, s, np.zeros(10), fixed=kin)
        assert O.lagrangian(qp, 0.0, x, mu) - phistar <= eps_in


@pytest.mark.parametrize("rho", [0.0, 0.5])
def test_inner_certificates_bound_suboptimality(rho):
    """Both inner certificates (FW gap, gradient-mapping bound with sigma = lmin(Q)) are upper
    bounds on L_rho(x, mu) - d_rho(mu), the quantity eq. duquad_in bounds by eps_in, and vanish
    at the inner minimiser."""
    inst, qp = _small(24, n=9, p=6, g_scale=0.02, box=0.5)
    mu = np.abs(np.random.default_rng(3).standard_normal(6))
    LL = inst.lmax_Q + rho * np.linalg.norm(inst.G, 2) ** 2
    xstar, _, _ = O.fom(qp, rho, mu, LL, inst.lmin_Q, np.zeros(9), fixed=30000)
    phistar = O.lagrangian(qp, rho, xstar, mu)
    rng = np.random.default_rng(4)
    for t in range(20):
        x = np.clip(xstar + rng.standard_normal(9) * 10.0 ** -rng.uniform(0, 6), -0.5, 0.5)
        sub = O.lagrangian(qp, rho, x, mu) - phistar
        assert O.fw_gap(qp, rho, x, mu) >= sub - 1e-13
        assert O.inner_cert(qp, rho, x, mu, LL, inst.lmin_Q) >= sub - 1e-13
    assert O.inner_cert(qp, rho, xstar, mu, LL, inst.lmin_Q) < 1e-12
    assert O.fw_gap(qp, rho, xstar, mu) < 1e-12
    assert O.inner_cert(qp, rho, xstar, mu, LL, 0.0) == O.fw_gap(qp, rho, xstar, mu)


@pytest.mark.parametrize("rho", [0.0, 0.5])
def test_step_certificate_bounds_suboptimality_of_the_step(rho):
    """The step certificate of y -> x+ = [y - grad/L]_U bounds L_rho(x+, mu) - d_rho(mu) for
    step points y inside and outside the box, vanishes at the inner minimiser, and its x+ is
    the inner iterate the FOM step produces (FOM started at y with GM for one step)."""
    inst, qp = _small(24, n=9, p=6, g_scale=0.02, box=0.5)
    mu = np.abs(np.random.default_rng(3).standard_normal(6))
    LL = inst.lmax_Q + rho * np.linalg.norm(inst.G, 2) ** 2
    xstar, _, _ = O.fom(qp, rho, mu, LL, inst.lmin_Q, np.zeros(9), fixed=30000)
    assert O.fw_gap(qp, rho, xstar, mu) < 1e-12   # x* is the minimiser over the box
    phistar = O.lagrangian(qp, rho, xstar, mu)
    rng = np.random.default_rng(5)
    tight = 0
    for t in range(40):
        y = xstar + rng.standard_normal(9) * 10.0 ** -rng.uniform(0, 6)
        if t % 2:
            y = np.clip(y, -0.5, 0.5)
        b, xp = O.step_cert(qp, rho, y, mu, LL, inst.lmin_Q)
        x1, _, _ = O.fom(qp, rho, mu, LL, inst.lmin_Q, y, fixed=1, variant=O.INNER_GM)
        np.testing.assert_allclose(xp, x1, rtol=0, atol=1e-15)
        assert np.all(xp >= -0.5) and np.all(xp <= 0.5)
        sub = O.lagrangian(qp, rho, xp, mu) - phistar
        assert b >= sub - 1e-13
        tight += b <= 1e3 * max(sub, 1e-16)
    assert tight > 0                               # not vacuous: within 1e3 of the true gap somewhere
    b, xp = O.step_cert(qp, rho, xstar, mu, LL, inst.lmin_Q)
    assert b < 1e-20 and np.allclose(xp, xstar, atol=1e-12)


@pytest.mark.parametrize("alg", ALGS)
def test_step_certificate_run_matches_kkt(alg):
    """DFOM whose inner loops stop on the step certificate reaches the brute-force KKT point."""
    inst, qp = _small(2, n=5, p=4, g_scale=0.02, box=0.3)
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    r = O.dfom(qp, alg, c, eps_in=1e-12, eps_out=1e-8, max_outer=400000, inner_cert_step=True)
    assert r.status == 0
    np.testing.assert_allclose(r.x_last, xs, atol=1e-3)
    assert abs(r.f_last - fs) <= 1e-7 + 1e-6 * abs(fs)
    assert r.d_lb <= fs + 1e-10
    eps = 1e-3
    r = O.dfom(qp, alg, c, eps_in=O.default_eps_in(alg, eps, c.Ld), eps_out=eps, max_outer=100000,
               inner_cert_step=True)
    assert r.status == 0
    if r.converged_last:
        assert r.infeas_last <= eps and r.f_last - fs <= eps
    if r.converged_avg:
        assert r.infeas_avg <= eps and r.f_avg - fs <= eps


# --------------------------------------------------------------- theory mode (Sec. 4-5)

def _theory_counts(qp, alg, inst, eps, Rd, rho=None):
    c = O.constants(qp, alg, rho=rho, lmin_Q=inst.lmin_Q)
    D_U = float(np.linalg.norm(inst.ub - inst.lb))
    ein = O.default_eps_in(alg, eps, c.Ld, Rd)
    kout = max(1, math.ceil(O.k_out(alg, eps, c.Ld, Rd)))
    kin = max(1, math.ceil(O.k_in(c.LL, c.sigma, D_U, ein)))
    return c, kout, kin


@pytest.mark.parametrize("alg", ALGS)
def test_theory_counts_meet_the_primal_bounds(alg):
    """With eps_in, k_out of eq. choose_ein, the FOM count k_in of Sec. 5 and lambda^0 = 0, the
    averaged primal output satisfies the theorems' bounds: (A)DGM dist_K <= eps / R_d and
    -eps <= F - F* <= eps / 4; (A)DFGM dist_K <= 3 eps / R_d and -3 eps <= F - F* <= 5 eps / 4.
    R_d = ||lambda*|| and F* come from brute-force KKT; ADGM/ADFGM use rho* = 8 R_d^2 / eps."""
    eps = 1e-2
    checked = 0
    for seed in range(1, 30):
        inst, qp = _small(seed, n=5, p=4, g_scale=0.02, box=0.3)
        xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
        Rd = float(np.linalg.norm(lam_s))
        if Rd < 0.1:
            continue                      # constraints inactive: nothing to certify
        rho = O.rho_star(eps, Rd) if alg in (O.ADGM, O.ADFGM) else None
        c, kout, kin = _theory_counts(qp, alg, inst, eps, Rd, rho)
        r = O.dfom(qp, alg, c, inner_fixed=kin, outer_fixed=kout)
        fast = alg in (O.DFGM, O.ADFGM)
        assert r.infeas_avg <= (3.0 if fast else 1.0) * eps / Rd
        assert -(3.0 if fast else 1.0) * eps <= r.f_avg - fs <= (1.25 if fast else 0.25) * eps
        checked += 1
        if checked == 3:
            break
    assert checked == 3


def test_rho_star_minimises_the_total_count():
    """k_out k_in as a function of rho (sigma = 0, the case the optimum is derived for; at
    least one outer iteration) is smallest at rho* = 8 R_d^2 / eps among a log-spaced sweep:
    below it the product falls like rho^{-1/4}, above it k_out = 1 and k_in grows."""
    inst, qp = _small(3, n=5, p=4, g_scale=0.02, box=0.3)
    eps, Rd = 1e-3, 1.5
    D_U = float(np.linalg.norm(inst.ub - inst.lb))
    normG2 = float(np.linalg.norm(inst.G, 2) ** 2)
    lmax = float(np.linalg.eigvalsh(inst.Q)[-1])

    def total(rho):
        LL, Ld = lmax + rho * normG2, normG2 / (rho * normG2)      # lambda_min taken as 0
        ein = O.default_eps_in(O.ADFGM, eps, Ld, Rd)
        return max(1.0, O.k_out(O.ADFGM, eps, Ld, Rd)) * O.k_in(LL, 0.0, D_U, ein)
    rhos = O.rho_star(eps, Rd) * np.logspace(-3, 3, 61)
    best = rhos[int(np.argmin([total(r) for r in rhos]))]
    assert 0.7 <= best / O.rho_star(eps, Rd) <= 1.5


@pytest.mark.parametrize("rho,cone", [(0.0, O.CONE_INEQ), (0.7, O.CONE_INEQ), (0.7, O.CONE_EQ)])
def test_sampled_step_matches_the_c_oracle(rho, cone):
    """The sampled FOM step (numpy, used at full size) equals one GM step of the C oracle from
    the same point, at every coordinate and at a sampled subset."""
    inst, _ = _small(8, n=9, p=6, g_scale=0.02, box=0.5)
    qp = _qp(inst, cone)
    rng = np.random.default_rng(2)
    y = rng.uniform(-0.5, 0.5, 9)
    mu = np.abs(rng.standard_normal(6)) if cone == O.CONE_INEQ else rng.standard_normal(6)
    LL = 40.0
    x1, _, _ = O.fom(qp, rho, mu, LL, 0.0, y, fixed=1, variant=O.INNER_GM)
    full = O.sampled_fom_step(q=inst.q, g=inst.g, G=inst.G, Q_rows=None, rows=None, y=y, mu=mu, rho=rho,
                              L=LL, lb=inst.lb, ub=inst.ub, Qy_full=inst.Q @ y, cone=cone)
    np.testing.assert_allclose(full, x1, rtol=0, atol=1e-14)
    rows = np.array([0, 3, 4, 8])
    part = O.sampled_fom_step(q=inst.q, g=inst.g, G=inst.G, Q_rows=inst.Q[rows], rows=rows, y=y, mu=mu,
                              rho=rho, L=LL, lb=inst.lb, ub=inst.ub, cone=cone)
    np.testing.assert_allclose(part, x1[rows], rtol=0, atol=1e-14)


# ------------------------------------------ the last primal iterate (eq. last_primal, Sec. 4.1)

def _dual_value_lbfgsb(qp, rho, lam):
    """d_rho(lam) = min over the box of L_rho(., lam) (eq. dual_fc) by scipy's L-BFGS-B: a route
    that shares nothing with Algorithm FOM (value and gradient of eq. auglag1 are pinned above
    against the minimum over s and against finite differences)."""
    from scipy.optimize import minimize
    f = lambda u: O.lagrangian(qp, rho, u, lam)
    jac = lambda u: O.grad_lagr(qp, rho, u, lam)
    best = None
    for x0 in (np.zeros(qp.n), 0.5 * (qp.lb + qp.ub) + 0.25 * (qp.ub - qp.lb)):
        m = minimize(f, x0, jac=jac, bounds=list(zip(qp.lb, qp.ub)), method="L-BFGS-B",
                     options=dict(ftol=1e-16, gtol=1e-13, maxiter=20000, maxcor=30))
        if best is None or m.fun < best.fun:
            best = m
    return float(best.fun), best.x


def _lambda_after(qp, alg, c, k, **kw):
    """lambda^k of Algorithm DFOM (lambda^0 = 0 for k = 0)."""
    if k == 0:
        return np.zeros(qp.p)
    return O.dfom(qp, alg, c, outer_fixed=k, want_avg=False, **kw).lam


def _active_instance(seed=31):
    # constraints active at the optimum and the box partly active, so lambda^k moves over
    # many outer iterations and ubar(lambda^k) differs from ubar(mu^k) far from convergence
    inst, qp = _small(seed, n=6, p=5, g_scale=0.02, box=0.4)
    return inst, qp


@pytest.mark.parametrize("alg", [O.DFGM, O.ADFGM])
def test_fast_last_iterate_solves_the_inner_problem_at_lambda_k(alg):
    """eq. last_primal for DFGM/ADFGM: the last primal output is ubar(lambda^k), an
    eps_in-solution (eq. duquad_in) of the inner problem at the last dual iterate lambda^k,
    not the chain iterate ubar^k = ubar(mu^k).  Checked far from convergence against d_rho
    from L-BFGS-B, with mu^k = lambda^{k-1} + beta_{k-1} (lambda^{k-1} - lambda^{k-2})."""
    inst, qp = _active_instance()
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    eps_in = 1e-7
    kw = dict(eps_in=eps_in, max_inner=200000)
    checked = 0
    for k in (3, 5, 8):
        r = O.dfom(qp, alg, c, outer_fixed=k, want_avg=False, trace_cap=k, **kw)
        ru = O.dfom(qp, alg, c, outer_fixed=k, want_last=False, **kw)   # x_last = ubar^k then
        lam_k = r.lam
        np.testing.assert_array_equal(lam_k, ru.lam)                      # the extra solve leaves the chain alone
        lam_1, lam_2 = _lambda_after(qp, alg, c, k - 1, **kw), _lambda_after(qp, alg, c, k - 2, **kw)
        mu_k = lam_1 + r.trace[k - 2, 3] * (lam_1 - lam_2)
        d_lam, _ = _dual_value_lbfgsb(qp, c.rho, lam_k)
        d_mu, _ = _dual_value_lbfgsb(qp, c.rho, mu_k)
        sub_last = O.lagrangian(qp, c.rho, r.x_last, lam_k) - d_lam
        assert -1e-10 <= sub_last <= eps_in + 1e-10
        assert O.inner_cert(qp, c.rho, r.x_last, lam_k, c.LL, c.sigma) <= eps_in
        # ubar^k solves the inner problem at mu^k, and is far from solving it at lambda^k
        assert O.lagrangian(qp, c.rho, ru.x_last, mu_k) - d_mu <= eps_in + 1e-10
        assert O.lagrangian(qp, c.rho, ru.x_last, lam_k) - d_lam > 100 * eps_in
        # and the last output is not an eps_in-solution at mu^k
        assert O.lagrangian(qp, c.rho, r.x_last, mu_k) - d_mu > 100 * eps_in
        checked += 1
    assert checked == 3


@pytest.mark.parametrize("alg", [O.DGM, O.ADGM])
def test_dgm_last_iterate_is_the_chain_iterate(alg):
    """eq. last_primal for DGM/ADGM: mu^{k+1} = lambda^k (beta = 0), so the last primal iterate
    is the inner solution the chain computes, ubar^k, with no extra solve."""
    inst, qp = _active_instance()
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    for k in (1, 4, 9):
        r = O.dfom(qp, alg, c, eps_in=1e-7, outer_fixed=k, want_avg=False)
        ru = O.dfom(qp, alg, c, eps_in=1e-7, outer_fixed=k, want_last=False)
        np.testing.assert_array_equal(r.x_last, ru.x_last)
        assert r.inner_iters == ru.inner_iters


@pytest.mark.parametrize("alg", [O.DFGM, O.ADFGM])
def test_fast_last_iterate_warm_starts_from_ubar_k(alg):
    """The extra inner solve of eq. last_primal is Algorithm FOM at mu = lambda^k started from
    ubar^k (the warm start of Sec. 3): with one inner iteration it is the projected gradient
    step [ubar^k - grad_u L_rho(ubar^k, lambda^k) / L_L]_U.  Starting it from 0, from
    ubar^{k-1} or taking the gradient at mu^k gives other points, which this separates."""
    inst, qp = _active_instance()
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    for k in (2, 6):
        r = O.dfom(qp, alg, c, inner_fixed=1, outer_fixed=k, want_avg=False, trace_cap=k)
        ubar_k = O.dfom(qp, alg, c, inner_fixed=1, outer_fixed=k, want_last=False).x_last
        ubar_km1 = O.dfom(qp, alg, c, inner_fixed=1, outer_fixed=k - 1, want_last=False).x_last
        lam_k = r.lam
        lam_1 = _lambda_after(qp, alg, c, k - 1, inner_fixed=1)
        lam_2 = _lambda_after(qp, alg, c, k - 2, inner_fixed=1)
        mu_k = lam_1 + r.trace[k - 2, 3] * (lam_1 - lam_2)

        def step(x, lam):
            return np.clip(x - O.grad_lagr(qp, c.rho, x, lam) / c.LL, qp.lb, qp.ub)
        np.testing.assert_allclose(r.x_last, step(ubar_k, lam_k), rtol=0, atol=1e-14)
        for wrong in (step(np.zeros(qp.n), lam_k), step(ubar_km1, lam_k), step(ubar_k, mu_k)):
            assert np.max(np.abs(wrong - r.x_last)) > 1e-6


@pytest.mark.parametrize("alg", ALGS)
def test_last_iterate_feasibility_and_suboptimality_links(alg):
    """Sec. 4.1, proof of the last-iterate theorem, at every k for the multiplier lam at which
    the last output ubar(lam) was computed (lam = lambda^k for (A)DFGM, mu^k = lambda^{k-1} for
    (A)DGM), with F*, lambda* from brute-force KKT and d_rho(lam) from L-BFGS-B:
      eq. aux_feas_bound   dist_K(G u + g) <= sqrt(2 L_d eps_in) + sqrt(2 L_d (F* - d(lam)))
      eq. aux_subopt_right F(u) - F* <= ||lam|| (sqrt(2 L_d eps_in) + sqrt(2 L_d (F* - d(lam)))) + eps_in
      eq. psubopt_left     F(u) - F* >= -||lambda*|| dist_K(G u + g)."""
    inst, qp = _active_instance()
    xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
    assert np.linalg.norm(lam_s) > 0.1                    # the instance has active constraints
    c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
    eps_in = 1e-6
    fast = alg in (O.DFGM, O.ADFGM)
    tight = 0
    for k in (1, 2, 4, 8, 16, 32):
        r = O.dfom(qp, alg, c, eps_in=eps_in, outer_fixed=k, want_avg=False, max_inner=200000)
        lam = r.lam if fast else _lambda_after(qp, alg, c, k - 1, eps_in=eps_in, max_inner=200000)
        d_lam, _ = _dual_value_lbfgsb(qp, c.rho, lam)
        gap = max(fs - d_lam, 0.0)
        inf = O.infeas(qp, r.x_last)
        link = math.sqrt(2 * c.Ld * eps_in) + math.sqrt(2 * c.Ld * gap)
        assert inf <= link + 1e-9
        assert r.f_last - fs <= np.linalg.norm(lam) * link + eps_in + 1e-9
        assert r.f_last - fs >= -np.linalg.norm(lam_s) * inf - 1e-9
        tight += inf >= 0.05 * link
    assert tight > 0                                       # the feasibility link is not vacuous here


@pytest.mark.parametrize("alg", [O.DGM, O.DFGM])
def test_last_iterate_theorem_at_k_out(alg):
    """The last-iterate theorem (Sec. 4.1, eq. pfeas_subopt_final and the |F - F*| bound after
    it): with eps_in and k_out of eq. choose_ein (R_d = ||lambda*||, lambda^0 = 0), ubar(lambda^k_out)
    satisfies dist_K <= max{(L_d eps)^{1/2}/sqrt(2), L_d^{1/4} eps^{3/4}/(3 R_d)^{1/2}} + (2 L_d eps)^{1/2}
    and |F - F*| <= 4 R_d max{...} + 4 R_d (2 L_d eps)^{1/2} + eps_in, given F* - d(lambda^k_out) <= eps."""
    eps = 1e-3
    checked = 0
    for seed in range(31, 60):
        inst, qp = _small(seed, n=6, p=5, g_scale=0.02, box=0.4)
        xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
        Rd = float(np.linalg.norm(lam_s))
        if Rd < 0.1:
            continue
        c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
        ein = O.default_eps_in(alg, eps, c.Ld, Rd)
        kout = max(1, math.ceil(O.k_out(alg, eps, c.Ld, Rd)))
        r = O.dfom(qp, alg, c, eps_in=ein, outer_fixed=kout, want_avg=False, max_inner=200000)
        lam = r.lam if alg == O.DFGM else _lambda_after(qp, alg, c, kout - 1, eps_in=ein, max_inner=200000)
        d_lam, _ = _dual_value_lbfgsb(qp, c.rho, lam)
        assert fs - d_lam <= eps                          # eq. bound_gen_dfg at k_out
        m = max(math.sqrt(c.Ld * eps) / math.sqrt(2.0), c.Ld ** 0.25 * eps ** 0.75 / math.sqrt(3.0 * Rd))
        feas = m + math.sqrt(2.0 * c.Ld * eps)
        assert O.infeas(qp, r.x_last) <= feas
        assert abs(r.f_last - fs) <= 4.0 * Rd * m + 4.0 * Rd * math.sqrt(2.0 * c.Ld * eps) + ein
        checked += 1
        if checked == 3:
            break
    assert checked == 3


@pytest.mark.parametrize("alg", ALGS)
@pytest.mark.parametrize("want", ["last", "avg"])
def test_fstar_stop_is_the_first_outer_meeting_the_papers_criterion(alg, want):
    """Sec. 6 stops on |F(u) - F*| <= eps and dist_K(Gu + g) <= eps with F* known: with F* from
    brute-force KKT the run stops at the first outer iteration whose output meets both (the run
    one iteration shorter does not), and the returned output meets them when re-scored."""
    eps = 1e-2
    done = 0
    for seed in range(1, 30):
        inst, qp = _small(seed, n=6, p=4, g_scale=0.02, box=0.3)
        xs, lam_s, fs = solve_kkt(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)
        c = O.constants(qp, alg, lmin_Q=inst.lmin_Q)
        kw = dict(eps_out=eps, eps_in=O.default_eps_in(alg, eps, c.Ld), max_outer=100000,
                  want_last=want == "last", want_avg=want == "avg")
        r = O.dfom(qp, alg, c, f_star=fs, **kw)
        assert r.status == 0
        x = r.x_last if want == "last" else r.x_avg
        assert abs(O.F(qp, x) - fs) <= eps and O.infeas(qp, x) <= eps
        if r.outer_iters < 2:
            continue
        prev = O.dfom(qp, alg, c, outer_fixed=r.outer_iters - 1, **kw)
        xp = prev.x_last if want == "last" else prev.x_avg
        assert abs(O.F(qp, xp) - fs) > eps or O.infeas(qp, xp) > eps
        # the certificate criterion is the stricter one (F - d_lb >= F - F*): never earlier
        rc = O.dfom(qp, alg, c, **kw)
        assert rc.outer_iters >= r.outer_iters
        done += 1
        if done == 2:
            break
    assert done == 2
