"""The seeded generators produce the structure their recipes state (host logic, no GPU):
spectra, feasibility, the MPC condensing identities, the uneven mix and the Poisson stream."""
import numpy as np
import pytest

import workloads as W


def test_single_dense_spectrum_and_signs():
    inst = W.single_dense(n=40, p=20, seed=0)
    ev = np.linalg.eigvalsh(inst.Q)
    assert np.allclose(inst.Q, inst.Q.T)
    assert ev[0] >= 1.0 - 1e-9 and ev[-1] <= 100.0 + 1e-9
    assert abs(ev[0] - inst.lmin_Q) <= 1e-9 * ev[-1] and abs(ev[-1] - inst.lmax_Q) <= 1e-9 * ev[-1]
    assert np.all(inst.g <= -0.1)                 # x = 0 strictly feasible
    assert np.all(inst.lb == -1.0) and np.all(inst.ub == 1.0)
    k = W.single_dense(n=30, p=15, seed=4, kappa=1e3)
    ev = np.linalg.eigvalsh(k.Q)
    assert abs(ev[0] - 1.0) <= 1e-9 and abs(ev[-1] - 1e3) <= 1e-6
    # the same seed gives the same instance
    assert np.array_equal(W.single_dense(n=40, p=20, seed=0).Q, inst.Q)


def test_haar_is_orthogonal():
    U = W.haar(np.random.default_rng(1), 25)
    assert np.allclose(U.T @ U, np.eye(25), atol=1e-12)


def test_large_dense_lambda_min_bound():
    d = W.large_dense(n=300, p=150, seed=1)
    Q = d["Q"].double().numpy()
    assert np.allclose(Q, Q.T)
    assert np.linalg.eigvalsh(Q)[0] >= d["lmin_Q"] - 1e-12
    assert (d["g"].double().numpy() <= -0.1).all()
    e = W.large_dense(n=300, p=150, seed=1, equality=True)
    G, g = e["G"].double().numpy(), e["g"].double().numpy()
    # g = -G u0 (u0 drawn inside the box): G u + g = 0 is solvable
    u, *_ = np.linalg.lstsq(G, -g, rcond=None)
    assert np.abs(G @ u + g).max() < 1e-10


def test_equality_dense_singular_and_feasible():
    inst = W.equality_dense(n=60, p=20, seed=3, n_zero=7)
    ev = np.linalg.eigvalsh(inst.Q)
    assert np.sum(np.abs(ev) < 1e-10) == 7 and inst.lmin_Q == 0.0
    assert inst.meta["cone"] == 1
    # the draw's u0 satisfies G u0 + g = 0 with |u0| <= 1/2: rebuild it from the same stream
    rng = np.random.default_rng(3)
    W.haar(rng, 60)
    rng.uniform(1.0, 100.0, 60)
    rng.standard_normal(60)
    rng.standard_normal((20, 60))
    u0 = rng.uniform(-0.5, 0.5, 60)
    assert np.abs(inst.G @ u0 + inst.g).max() < 1e-12


def test_mpc_condensing_matches_simulation():
    m = W.mpc_matrices(nx=4, nu=2, N=6, seed=2)
    A, B = m["A"], m["B"]
    assert abs(np.max(np.abs(np.linalg.eigvals(A))) - 0.95) < 1e-12
    rng = np.random.default_rng(0)
    x0, u = rng.standard_normal(4), rng.standard_normal(12)
    x, xs = x0.copy(), []
    for k in range(6):             # x_{k+1} = A x_k + B u_k
        x = A @ x + B @ u[2 * k:2 * k + 2]
        xs.append(x)
    assert np.allclose(np.concatenate(xs), m["Phi"] @ x0 + m["Gamma"] @ u, atol=1e-12)


def test_mpc_batch_shares_matrices_and_u0_feasible():
    d = W.mpc_batch(batch=64, nx=4, nu=2, N=6, seed=2)
    Q, G, qs, gs = d["Q"], d["G"], d["qs"], d["gs"]
    assert Q.shape == (12, 12) and G.shape == (48, 12) and qs.shape == (64, 12) and gs.shape == (64, 48)
    assert np.linalg.eigvalsh(Q)[0] >= d["lmin_Q"] - 1e-12    # Gamma' Gamma + 0.1 I
    assert np.all(gs < 0)                                       # u = 0 strictly feasible
    m = W.mpc_matrices(nx=4, nu=2, N=6, seed=2)
    # state bounds |x_k| <= b: G u + g <= 0  <=>  -b <= Phi x0 + Gamma u <= b
    x0, u = d["x0s"][5], np.zeros(12)
    sim = m["Phi"] @ x0 + m["Gamma"] @ u
    assert np.allclose(G @ u + gs[5], np.concatenate([sim - d["b"], -sim - d["b"]]))


def test_uneven_mix():
    ns, kappas, algs, seeds = W.uneven_sizes(count=5000, seed=3)
    assert ns.min() >= 16 and ns.max() <= 512
    assert kappas.min() >= 10.0 and kappas.max() <= 1e4
    assert set(np.unique(algs)) == {0, 1, 2, 3}
    inst = W.uneven_instance(ns[0], kappas[0], algs[0], seeds[0])
    assert inst.p == inst.n // 2 and inst.alg == W.ALGS[int(algs[0])]
    ev = np.linalg.eigvalsh(inst.Q)
    assert abs(ev[0] - 1.0) < 1e-8 and abs(ev[-1] - kappas[0]) < 1e-8 * kappas[0]


def test_served_stream_is_poisson():
    t, kinds, picks = W.served_stream(rate=2000.0, duration=5.0, seed=4, mpc_fraction=0.05)
    assert np.all(np.diff(t) > 0) and t[-1] < 5.0
    assert abs(t.size - 10000) < 4 * np.sqrt(10000)                        # Poisson count, 4 sigma
    gaps = np.diff(t)
    assert abs(gaps.mean() - 1 / 2000.0) < 0.05 / 2000.0
    assert abs(kinds.mean() - 0.05) < 0.02


def test_hidden_top_eigenvectors_are_orthogonal_to_ones():
    """The hidden-top generator: Q's and G'G's top eigenvectors are +-(1, -1, 0, ...)/sqrt(2),
    orthogonal to the all-ones vector, with the stated eigenvalues; Q is symmetric."""
    inst = W.hidden_top(n=60, p=25, seed=3)
    v = np.zeros(60)
    v[:2] = (1.0, -1.0)
    v /= np.sqrt(2.0)
    ev, U = np.linalg.eigh(inst.Q)
    assert np.array_equal(inst.Q, inst.Q.T)
    assert abs(ev[-1] - 200.0) <= 1e-9 * 200 and ev[-2] <= 100.0 + 1e-9
    assert abs(abs(U[:, -1] @ v) - 1.0) <= 1e-12 and abs(U[:, -1].sum()) <= 1e-10
    eg, V = np.linalg.eigh(inst.G.T @ inst.G)
    assert abs(eg[-1] - 9.0) <= 1e-9 and eg[-2] <= 1.0 + 1e-12
    assert abs(abs(V[:, -1] @ v) - 1.0) <= 1e-12
    assert inst.lmin_Q <= ev[0] and ev[0] >= 1.0 - 1e-9


def test_sparse_qp_is_valid_csr_and_symmetric_pd():
    """The sparse generator: valid CSR (offsets, strictly increasing columns), Q symmetric with
    lambda_min(Q) >= 1 (Laplacian + diag >= 1), G with row_nnz distinct columns per row, and the
    dense expansion equal to the CSR arrays."""
    d = W.sparse_qp(n=300, p=120, deg=8, row_nnz=8, seed=3, dense=True)
    n, p = 300, 120
    for pre, rows in (("Q", n), ("G", p)):
        rp, ci = d[pre + "_rowptr"], d[pre + "_col"]
        assert rp.dtype == np.int32 and ci.dtype == np.int32 and rp[0] == 0 and rp[-1] == ci.size
        for r in range(rows):
            c = ci[rp[r]:rp[r + 1]]
            assert np.all(np.diff(c) > 0) and c.min() >= 0 and c.max() < n
    Q, G = d["Q"], d["G"]
    assert np.array_equal(Q, Q.T)
    assert np.linalg.eigvalsh(Q)[0] >= 1.0 - 1e-9
    assert np.all(np.diff(d["G_rowptr"]) == 8) and np.count_nonzero(G) == p * 8
    x = np.random.default_rng(0).standard_normal(n)
    Qx = np.array([d["Q_val"][d["Q_rowptr"][r]:d["Q_rowptr"][r + 1]] @ x[d["Q_col"][d["Q_rowptr"][r]:d["Q_rowptr"][r + 1]]]
                   for r in range(n)])
    np.testing.assert_allclose(Qx, Q @ x, rtol=1e-12, atol=1e-12)
    assert np.all(d["g"] <= -0.1)
