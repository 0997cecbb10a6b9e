"""GPU tests of the Lipschitz estimates, input validation and failure detection, through the C ABI.

Lipschitz constants (Sec. 3 Step 1 and eq. Ld): Algorithm FOM's step 1/L_L and both inner
certificates need L_L and ||G||^2 to be upper bounds.  The Lanczos estimate starts from a
pseudo-random vector, so a Q or G'G whose top eigenvector is orthogonal to the all-ones vector
cannot hide it; the DQ_LIP_BOUND mode gives guaranteed bounds.  Validation: non-finite values,
lb > ub and an asymmetric Q are refused on the device at dq_problem_create / set_vectors.
Failure detection: an infeasible QP ends with DQ_ERR_DIVERGED once the certified dual lower
bound passes the largest value F takes on the box (weak duality), and a bounded device-side
wait that runs out returns DQ_ERR_TIMEOUT with the context still usable.
"""
import ctypes

import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import ALG_IDS, exact_constants, gpu_problem, oracle_qp

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


def _rescored(inst, alg, x, eps):
    """FP64 re-scoring by the oracle: infeasibility and the gap to a certified lower bound on F*."""
    qp = oracle_qp(inst)
    c = exact_constants(inst, alg)
    ref = O.dfom(qp, ALG_IDS[alg], c, eps_out=eps * 0.01, eps_in=1e-10, max_outer=50000)
    return O.infeas(qp, x), O.F(qp, x) - ref.d_lb


@pytest.mark.parametrize("prec_name", ["FP32", "FP64"])
@pytest.mark.parametrize("engine_name,n,p", [("CTA", 60, 30), ("CTA", 200, 80), ("GRID", 600, 300)])
def test_lanczos_finds_a_top_eigenvector_orthogonal_to_ones(ctx, engine_name, n, p, prec_name):
    """lambda_max(Q) = 200 and ||G||^2 = 9 along (1, -1, 0, ...)/sqrt(2), the rest of the spectra
    at most 100 and 1: the estimates are upper bounds within 2 %, and the certified FP32/FP64
    solve they drive is eps-optimal when re-scored by the oracle in FP64.  n = 60, p = 30 in FP32
    takes the thread-block engine's one-warp Lanczos, the other cases its block version."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.hidden_top(n=n, p=p, seed=n)
    prec = getattr(D, prec_name)
    engine = getattr(D, "ENGINE_" + engine_name)
    P = gpu_problem(ctx, inst, prec)
    eps = 1e-3
    xl, xa, lam, (r,) = P.solve(D.opts("ADFGM", eps_out=eps, max_outer=5000, engine=engine))
    lmax, _, nG2 = P.constants()
    lt = np.linalg.eigvalsh(inst.Q)[-1]
    gt = np.linalg.norm(inst.G, 2) ** 2
    assert lt <= lmax <= 1.02 * lt, (lmax, lt)
    assert gt <= nG2 <= 1.02 * gt, (nG2, gt)
    assert r.status == 0
    x = xl if r.converged_last else xa
    inf, gap = _rescored(inst, "ADFGM", x, eps)
    assert inf <= eps * 1.01 and gap <= eps * 1.01, (inf, gap)


@pytest.mark.parametrize("n,p", [(50, 50), (61, 17), (300, 120)])
def test_paired_fp64_lanczos_equals_the_single_runs(ctx, n, p):
    """With both constants wanted, an FP64 thread-block solve runs the Q and G'G Lanczos
    iterations in one loop; each must return exactly what its run alone returns (the run alone
    is taken when the other constant is supplied)."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=n, p=p, seed=300 + n, lam_lo=1.0, lam_hi=100.0)
    o = D.opts("DFGM", fixed_outer=1, fixed_inner=1, engine=D.ENGINE_CTA)
    P = gpu_problem(ctx, inst, D.FP64)
    P.solve(o)
    lmax, _, nG2 = P.constants()
    P.close()
    Pq = gpu_problem(ctx, inst, D.FP64, normG2=nG2)
    Pq.solve(o)
    lmax_alone = Pq.constants()[0]
    Pq.close()
    Pg = gpu_problem(ctx, inst, D.FP64, lmax_Q=lmax)
    Pg.solve(o)
    nG2_alone = Pg.constants()[2]
    Pg.close()
    assert lmax == lmax_alone and nG2 == nG2_alone, (lmax, lmax_alone, nG2, nG2_alone)
    # upper bounds (the top of these spectra is clustered: theta + 2 r can sit several % above)
    assert lmax >= np.linalg.eigvalsh(inst.Q)[-1] * (1 - 1e-12)
    assert nG2 >= np.linalg.norm(inst.G, 2) ** 2 * (1 - 1e-12)


@pytest.mark.parametrize("engine_name,n,p", [("CTA", 120, 50), ("GRID", 400, 150)])
def test_guaranteed_bound_mode(ctx, engine_name, n, p):
    """DQ_LIP_BOUND: min(Gershgorin, Frobenius) and min(||G||_1 ||G||_inf, ||G||_F^2) are at
    least the true constants (and equal the FP64 formulas), and the solve stays eps-optimal."""
    from paper_1504_05708_gb300 import duquad as D
    inst = W.hidden_top(n=n, p=p, seed=7 + n)
    engine = getattr(D, "ENGINE_" + engine_name)
    P = gpu_problem(ctx, inst, D.FP64, lipschitz=D.LIP_BOUND)
    eps = 1e-3
    xl, xa, lam, (r,) = P.solve(D.opts("DFGM", eps_out=eps, max_outer=20000, engine=engine))
    lmax, _, nG2 = P.constants()
    A, G = inst.Q, inst.G
    b_q = min(np.abs(A).sum(axis=1).max(), np.linalg.norm(A, "fro"))
    b_g = min(np.abs(G).sum(axis=0).max() * np.abs(G).sum(axis=1).max(), np.linalg.norm(G, "fro") ** 2)
    assert abs(lmax - b_q) <= 1e-12 * b_q and abs(nG2 - b_g) <= 1e-12 * b_g
    assert lmax >= np.linalg.eigvalsh(A)[-1] and nG2 >= np.linalg.norm(G, 2) ** 2
    assert r.status == 0
    x = xl if r.converged_last else xa
    inf, gap = _rescored(inst, "DFGM", x, eps)
    assert inf <= eps * 1.01 and gap <= eps * 1.01, (inf, gap)


def _infeasible(n, seed):
    """x_1 <= -0.5 and x_1 >= 0.5 at once: no feasible point, the box is [-1, 1]^n."""
    inst = W.single_dense(n=n, p=2, seed=seed, lam_lo=1.0, lam_hi=2.0)
    G = np.zeros((2, n))
    G[0, 0], G[1, 0] = 1.0, -1.0
    inst.G = G
    inst.g = np.array([0.5, 0.5])
    return inst


@pytest.mark.parametrize("alg", ["DGM", "DFGM", "ADGM", "ADFGM"])
@pytest.mark.parametrize("engine_name,n", [("CTA", 12), ("GRID", 300)])
def test_infeasible_qp_diverges(ctx, engine_name, n, alg):
    from paper_1504_05708_gb300 import duquad as D
    inst = _infeasible(n, 11)
    P = gpu_problem(ctx, inst, D.FP64)
    with pytest.raises(D.DuquadError) as e:
        P.solve(D.opts(alg, eps_out=1e-3, max_outer=200000, engine=getattr(D, "ENGINE_" + engine_name)))
    assert e.value.status == D.ERR_DIVERGED
    # a feasible QP on the same context still solves
    ok = W.single_dense(n=n, p=2, seed=11, lam_lo=1.0, lam_hi=2.0)
    _, _, _, (r,) = gpu_problem(ctx, ok, D.FP64).solve(D.opts(alg, eps_out=1e-3,
                                                              engine=getattr(D, "ENGINE_" + engine_name)))
    assert r.status == 0


@pytest.mark.parametrize("device_arrays", [False, True])
@pytest.mark.parametrize("prec_name", ["FP32", "FP64"])
def test_asymmetric_Q_rejected(ctx, prec_name, device_arrays):
    import torch
    from paper_1504_05708_gb300 import duquad as D
    prec = getattr(D, prec_name)
    inst = W.single_dense(n=70, p=20, seed=4)
    bad = W.single_dense(n=70, p=20, seed=4)
    bad.Q[33, 5] += 1e-3 * np.sqrt(bad.Q[33, 33] * bad.Q[5, 5])

    def make(i):
        if not device_arrays:
            return gpu_problem(ctx, i, prec)
        dt = torch.float32 if prec == D.FP32 else torch.float64
        t = {k: torch.tensor(getattr(i, k), dtype=dt, device="cuda") for k in ("Q", "q", "G", "g", "lb", "ub")}
        return D.Problem(ctx, t["Q"], t["q"], t["G"], t["g"], t["lb"], t["ub"], prec=prec, lmin_Q=i.lmin_Q)

    with pytest.raises(D.DuquadError) as e:
        make(bad)
    assert e.value.status == D.ERR_INVALID and "symmetric" in str(e.value)
    make(inst).close()  # a symmetric Q (and its FP32 rounding) passes


def test_nonfinite_and_box_rejected_on_device(ctx):
    import torch
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=40, p=30, seed=2)
    for field, idx, val in (("Q", (3, 3), np.inf), ("G", (29, 39), np.nan), ("g", (0,), np.nan),
                            ("ub", (7,), np.nan)):
        b = W.single_dense(n=40, p=30, seed=2)
        getattr(b, field)[idx] = val
        for prec in (D.FP64, D.FP32):
            with pytest.raises(D.DuquadError) as e:
                gpu_problem(ctx, b, prec)
            assert e.value.status == D.ERR_INVALID
    b = W.single_dense(n=40, p=30, seed=2)
    b.lb[5] = 1.5
    with pytest.raises(D.DuquadError) as e:
        gpu_problem(ctx, b, D.FP32)
    assert "lb > ub" in str(e.value)
    # device arrays: the same checks run on the caller's memory
    t = {k: torch.tensor(getattr(inst, k), dtype=torch.float32, device="cuda") for k in ("Q", "q", "G", "g", "lb", "ub")}
    t["G"][4, 4] = float("nan")
    with pytest.raises(D.DuquadError):
        D.Problem(ctx, t["Q"], t["q"], t["G"], t["g"], t["lb"], t["ub"], prec=D.FP32, lmin_Q=inst.lmin_Q)


def test_set_vectors_rejects_nonfinite_and_keeps_the_old_ones(ctx):
    from paper_1504_05708_gb300 import duquad as D
    inst = W.single_dense(n=50, p=25, seed=0, g_scale=0.02)
    P = gpu_problem(ctx, inst, D.FP64)
    o = D.opts("DFGM", fixed_inner=10, fixed_outer=6, engine=D.ENGINE_CTA)
    xl0, _, _, _ = P.solve(o)
    q_bad = inst.q.copy()
    q_bad[10] = np.nan
    with pytest.raises(D.DuquadError) as e:
        P.set_vectors(q=q_bad, g=inst.g * 2.0)
    assert e.value.status == D.ERR_INVALID
    xl1, _, _, _ = P.solve(o)
    assert np.array_equal(xl0, xl1)
    P.set_vectors(q=-inst.q)
    xl2, _, _, _ = P.solve(o)
    assert not np.array_equal(xl0, xl2)


def test_bounded_wait_gives_up_and_context_survives(ctx):
    """The engines' mbarrier wait, polled against the GPU's global timer: with no arrival it gives
    up after the limit and the call returns DQ_ERR_TIMEOUT; the CUDA context stays usable."""
    import time

    import torch
    from paper_1504_05708_gb300 import duquad as D
    L = D.lib()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    assert L.dq_test_bounded_wait(2_000_000, 1, stream) == D.OK
    t0 = time.perf_counter()
    assert L.dq_test_bounded_wait(20_000_000, 0, stream) == D.ERR_TIMEOUT
    assert time.perf_counter() - t0 >= 0.015
    assert L.dq_test_bounded_wait(0, 0, stream) == D.ERR_INVALID
    torch.cuda.synchronize()
    inst = W.single_dense(n=50, p=25, seed=0, g_scale=0.02)
    _, _, _, (r,) = gpu_problem(ctx, inst, D.FP64).solve(D.opts("DFGM", eps_out=1e-4, engine=D.ENGINE_CTA))
    assert r.status == 0
