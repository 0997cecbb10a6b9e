"""dq_solve_noalloc: the allocation-free solve gives the same answer as dq_solve.

Callers that cannot allocate device memory while running (a real-time control
loop, or a process whose memory pool already holds the GPU) use this entry
point; it keeps its scratch in one fixed device array inside the library.  This
file is collected last so that a run stopping at the first failure has already
run every other test; it passes both alone in a fresh process and after them.
"""
import ctypes

import numpy as np
import pytest

import workloads as W
from gpu_helpers import exact_constants, gpu_opts_from, rel

pytestmark = pytest.mark.gpu


def _desc(D, t, inst, prec):
    d = D.ProblemDesc()
    d.n, d.p, d.batch, d.cone, d.prec, d.memory = inst.n, inst.p, 1, D.CONE_INEQ, prec, D.DEVICE
    d.Q, d.q, d.G, d.g = t["Q"].data_ptr(), t["q"].data_ptr(), t["G"].data_ptr(), t["g"].data_ptr()
    d.lb, d.ub = t["lb"].data_ptr(), t["ub"].data_ptr()
    d.lmax_Q, d.lmin_Q, d.normG2 = float("nan"), inst.lmin_Q, float("nan")
    return d


@pytest.mark.parametrize("prec_name,n,p,tol", [("FP64", 50, 25, 1e-9), ("FP32", 200, 100, 1e-6)])
def test_noalloc_matches_dq_solve_twice(prec_name, n, p, tol):
    import torch
    from paper_1504_05708_gb300 import duquad as D
    prec = getattr(D, prec_name)
    dt = torch.float64 if prec == D.FP64 else torch.float32
    inst = W.single_dense(n=n, p=p, seed=0, g_scale=0.02)
    t = {k: torch.tensor(getattr(inst, k), dtype=dt, device="cuda") for k in ("Q", "q", "G", "g", "lb", "ub")}
    c = exact_constants(inst, "DFGM")
    o = gpu_opts_from(c, "DFGM", eps_out=1e-4, engine=D.ENGINE_CTA)
    # the existing entry point
    ctx = D.Context(0)
    P = D.Problem(ctx, inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub, prec=prec, lmin_Q=inst.lmin_Q)
    xl_ref, xa_ref, lm_ref, (r_ref,) = P.solve(o)
    P.close()
    ctx.close()
    stream = ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)
    desc = _desc(D, t, inst, prec)
    # call 0 is the set-up call (it loads the library's kernels and the fixed array onto the
    # device under lazy module loading); calls 1 and 2 must allocate nothing, and the scratch
    # keeps the last call's contents, which a later call must not see
    for call in range(3):
        xl = torch.full((n,), float("nan"), dtype=dt, device="cuda")
        xa = torch.full((n,), float("nan"), dtype=dt, device="cuda")
        lm = torch.full((p,), float("nan"), dtype=dt, device="cuda")
        out = D.Outputs()
        out.x_last, out.x_avg, out.lambda_, out.memory = xl.data_ptr(), xa.data_ptr(), lm.data_ptr(), D.DEVICE
        res = D.Result()
        torch.cuda.synchronize()
        free0, _ = torch.cuda.mem_get_info(0)
        st = D.lib().dq_solve_noalloc(0, ctypes.byref(desc), ctypes.byref(o), ctypes.byref(out), ctypes.byref(res),
                                      stream)
        torch.cuda.synchronize()
        free1, _ = torch.cuda.mem_get_info(0)
        D.check(st)
        if call > 0:
            assert free1 == free0, (call, free0, free1)
        assert res.status == r_ref.status == 0
        assert (res.outer_iters, res.inner_iters) == (r_ref.outer_iters, r_ref.inner_iters)
        assert rel(xl.cpu().double().numpy(), xl_ref) <= tol
        assert rel(xa.cpu().double().numpy(), xa_ref) <= tol
        assert rel(lm.cpu().double().numpy(), lm_ref) <= tol or np.linalg.norm(lm_ref) == 0


def test_noalloc_rejects_oversized():
    import torch
    from paper_1504_05708_gb300 import duquad as D
    n, p = 2048, 1024  # n * p = 2 M doubles > the fixed scratch
    d = D.ProblemDesc()
    z = torch.zeros(8, dtype=torch.float64, device="cuda")
    d.n, d.p, d.batch, d.cone, d.prec, d.memory = n, p, 1, D.CONE_INEQ, D.FP64, D.DEVICE
    d.Q = d.q = d.G = d.g = d.lb = d.ub = z.data_ptr()
    d.lmax_Q, d.lmin_Q, d.normG2 = 1.0, 1.0, 1.0
    res = D.Result()
    st = D.lib().dq_solve_noalloc(0, ctypes.byref(d), ctypes.byref(D.opts("DFGM")), None, ctypes.byref(res), None)
    assert st == D.ERR_INVALID
    assert b"scratch" in D.lib().dq_last_error()
