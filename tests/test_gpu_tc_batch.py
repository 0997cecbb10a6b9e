"""Shared-matrix batches on the tensor cores (bf16 hi/lo operands, FP32 accumulation).

Parity bar for the split-precision path: every instance's output, re-scored in
FP64 by the oracle, is eps-optimal, and ||x - x_oracle|| / ||x_oracle|| <= 1e-3.
"""
import numpy as np
import pytest

import oracle as O
import workloads as W
from gpu_helpers import rel

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def ctx():
    from paper_1504_05708_gb300 import duquad as D
    c = D.Context(0)
    yield c
    c.close()


def _mpc(B, seed=2):
    d = W.mpc_batch(batch=B, seed=seed)
    return d


def _problem(ctx, d, prec):
    from paper_1504_05708_gb300 import duquad as D
    B = d["qs"].shape[0]
    return D.Problem(ctx, d["Q"], d["qs"], d["G"], d["gs"], d["lb"], d["ub"], prec=prec, batch=B,
                     lmin_Q=float(np.linalg.eigvalsh(d["Q"])[0]) * 0.999)


def test_fixed_counts_match_fp32_engine(ctx):
    """Same iteration counts: the tensor-core path tracks the FP32 CTA engine on every instance."""
    from paper_1504_05708_gb300 import duquad as D
    d = _mpc(300)  # three tiles, the last one partial
    o = D.opts("DFGM", fixed_inner=40, fixed_outer=6)
    Pt = _problem(ctx, d, D.BF16X3)
    Pf = _problem(ctx, d, D.FP32)
    xt, at, lt, rt = Pt.solve(o)
    xf, af, lf, rf = Pf.solve(D.opts("DFGM", fixed_inner=40, fixed_outer=6, engine=D.ENGINE_CTA))
    errs = [rel(xt[b], xf[b]) for b in range(300)]
    assert max(errs) <= 2e-3, max(errs)
    assert [(r.outer_iters, r.inner_iters) for r in rt] == [(r.outer_iters, r.inner_iters) for r in rf]


@pytest.mark.parametrize("alg", ["DGM", "DFGM"])
def test_mpc_eps_optimal_vs_oracle(ctx, alg):
    from paper_1504_05708_gb300 import duquad as D
    B = 130
    d = _mpc(B, seed=5)
    lmin = float(np.linalg.eigvalsh(d["Q"])[0]) * 0.999
    eps = 1e-3
    P = _problem(ctx, d, D.BF16X3)
    # DGM's O(L_d R_d^2 / eps) outer bound (Sec. 4) is far above DFGM's: give it room
    max_outer = 200000 if alg == "DGM" else 20000
    xl, xa, lam, res = P.solve(D.opts(alg, eps_out=eps, eps_in=1e-5, check_every=5, max_outer=max_outer))
    bad = [(b, r.status, r.outer_iters) for b, r in enumerate(res) if r.status != 0]
    assert not bad, bad[:10]
    for b in (0, 64, B - 1):
        qp = O.QP(d["Q"], d["qs"][b], d["G"], d["gs"][b], d["lb"], d["ub"])
        c = O.constants(qp, O.DFGM, lmin_Q=lmin)
        # FP64 reference; its d_lb bounds F* from below whether or not it converged
        ro = O.dfom(qp, O.DFGM, c, eps_in=1e-8, eps_out=1e-4, outer_check_every=10, max_outer=20000)
        x = xl[b] if res[b].converged_last else xa[b]
        assert O.infeas(qp, x) <= eps * 1.01
        assert O.F(qp, x) - ro.d_lb <= eps * 1.01
        assert rel(x, ro.x_last) <= 1e-3 or (not res[b].converged_last)


def test_alone_equals_in_batch(ctx):
    """An instance gives bit-identical output alone and inside a larger batch (columns of a
    tensor-core product are independent and its frozen lanes never change)."""
    from paper_1504_05708_gb300 import duquad as D
    d = _mpc(200, seed=7)
    o = D.opts("DFGM", eps_out=1e-3, eps_in=1e-5, check_every=5)
    Pb = _problem(ctx, d, D.BF16X3)
    xb, ab, lb, rb = Pb.solve(o)
    for b in (0, 77, 199):
        one = {k: v for k, v in d.items()}
        one["qs"] = np.vstack([d["qs"][b], d["qs"][b]])
        one["gs"] = np.vstack([d["gs"][b], d["gs"][b]])
        P1 = _problem(ctx, one, D.BF16X3)
        x1, a1, l1, r1 = P1.solve(o)
        assert np.array_equal(x1[0], xb[b])
        assert (r1[0].outer_iters, r1[0].inner_iters) == (rb[b].outer_iters, rb[b].inner_iters)


def test_rejects_unsupported(ctx):
    from paper_1504_05708_gb300 import duquad as D
    d = _mpc(4)
    P = _problem(ctx, d, D.BF16X3)
    with pytest.raises(D.DuquadError):
        P.solve(D.opts("ADFGM"))
