"""Thin ctypes binding of include/duquad.h (argument marshalling only).

Every computation runs in libduquad.so's CUDA kernels; this module converts
arguments, allocates nothing on the GPU itself and raises when the library
is missing or a call fails.  torch is used only to hand device pointers and
the current CUDA stream to the library.
"""
from __future__ import annotations

import ctypes
import math
import os
from dataclasses import dataclass

import numpy as np

from . import _build

DGM, DFGM, ADGM, ADFGM = 0, 1, 2, 3
ALGS = {"DGM": DGM, "DFGM": DFGM, "ADGM": ADGM, "ADFGM": ADFGM}
OUT_LAST, OUT_AVERAGE, OUT_BOTH = 1, 2, 3
FP64, FP32, BF16X3 = 0, 1, 2
INNER_GAP, INNER_FIXED = 0, 1
CERT_AUTO, CERT_POINT, CERT_STEP = 0, 1, 2
CONE_INEQ, CONE_EQ = 0, 1
LIP_LANCZOS, LIP_BOUND = 0, 1
HOST, DEVICE = 0, 1
ENGINE_AUTO, ENGINE_CTA, ENGINE_GRID, ENGINE_TC = 0, 1, 2, 3
OK, NOT_CONVERGED, PENDING = 0, 1, 2
ERR_INVALID, ERR_NOMEM, ERR_CUDA, ERR_NONFINITE, ERR_DIVERGED, ERR_TIMEOUT, ERR_REJECTED = -1, -2, -3, -4, -5, -6, -7

NAN = float("nan")


class ProblemDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32), ("batch", ctypes.c_int32),
                ("cone", ctypes.c_int32), ("prec", ctypes.c_int32), ("memory", ctypes.c_int32),
                ("Q", ctypes.c_void_p), ("q", ctypes.c_void_p), ("G", ctypes.c_void_p),
                ("g", ctypes.c_void_p), ("lb", ctypes.c_void_p), ("ub", ctypes.c_void_p),
                ("lmax_Q", ctypes.c_double), ("lmin_Q", ctypes.c_double), ("normG2", ctypes.c_double),
                ("lipschitz", ctypes.c_int32)]


class SparseDesc(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int32), ("p", ctypes.c_int32), ("cone", ctypes.c_int32), ("prec", ctypes.c_int32),
                ("memory", ctypes.c_int32), ("nnz_Q", ctypes.c_int32), ("nnz_G", ctypes.c_int32),
                ("Q_rowptr", ctypes.c_void_p), ("Q_col", ctypes.c_void_p), ("Q_val", ctypes.c_void_p),
                ("G_rowptr", ctypes.c_void_p), ("G_col", ctypes.c_void_p), ("G_val", ctypes.c_void_p),
                ("q", ctypes.c_void_p), ("g", ctypes.c_void_p), ("lb", ctypes.c_void_p), ("ub", ctypes.c_void_p),
                ("lmax_Q", ctypes.c_double), ("lmin_Q", ctypes.c_double), ("normG2", ctypes.c_double),
                ("lipschitz", ctypes.c_int32)]


class SolveOpts(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int32), ("output", ctypes.c_int32), ("inner_stop", ctypes.c_int32),
                ("engine", ctypes.c_int32), ("eps_out", ctypes.c_double), ("eps_in", ctypes.c_double),
                ("rho", ctypes.c_double), ("fixed_outer", ctypes.c_int32), ("fixed_inner", ctypes.c_int32),
                ("max_outer", ctypes.c_int32), ("max_inner", ctypes.c_int32),
                ("check_every", ctypes.c_int32), ("inner_check_every", ctypes.c_int32),
                ("warm_start", ctypes.c_int32), ("kd_literal", ctypes.c_int32),
                ("Ld", ctypes.c_double), ("LL", ctypes.c_double), ("sigma", ctypes.c_double),
                ("fresh_constants", ctypes.c_int32), ("inner_cert", ctypes.c_int32),
                ("stop_fstar", ctypes.c_int32), ("f_star", ctypes.c_double)]


class Result(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int32), ("outer_iters", ctypes.c_int32),
                ("inner_iters", ctypes.c_int64), ("converged_last", ctypes.c_int32),
                ("converged_avg", ctypes.c_int32), ("f_last", ctypes.c_double),
                ("infeas_last", ctypes.c_double), ("f_avg", ctypes.c_double),
                ("infeas_avg", ctypes.c_double), ("d_lb", ctypes.c_double), ("Ld", ctypes.c_double),
                ("LL", ctypes.c_double), ("sigma", ctypes.c_double), ("rho", ctypes.c_double),
                ("alpha", ctypes.c_double)]

    def asdict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class Outputs(ctypes.Structure):
    _fields_ = [("x_last", ctypes.c_void_p), ("x_avg", ctypes.c_void_p), ("lambda_", ctypes.c_void_p),
                ("memory", ctypes.c_int32)]


class TheoryIn(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int32), ("eps", ctypes.c_double), ("Rd", ctypes.c_double),
                ("D_U", ctypes.c_double), ("lmax_Q", ctypes.c_double), ("lmin_Q", ctypes.c_double),
                ("normG2", ctypes.c_double), ("rho", ctypes.c_double)]


class TheoryOut(ctypes.Structure):
    _fields_ = [("rho", ctypes.c_double), ("LL", ctypes.c_double), ("sigma", ctypes.c_double),
                ("Ld", ctypes.c_double), ("eps_in", ctypes.c_double), ("k_out", ctypes.c_int64),
                ("k_in", ctypes.c_int64), ("k_total", ctypes.c_int64)]


class TheorySolveOpts(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int32), ("eps", ctypes.c_double), ("Rd", ctypes.c_double),
                ("safety", ctypes.c_double), ("rho", ctypes.c_double), ("max_total", ctypes.c_int64),
                ("engine", ctypes.c_int32)]


class Stats(ctypes.Structure):
    _fields_ = [("launches", ctypes.c_int64), ("gemv_launches", ctypes.c_int64), ("gemv_ms", ctypes.c_double),
                ("gemv_bytes", ctypes.c_double), ("reduce_launches", ctypes.c_int64),
                ("reduce_ms", ctypes.c_double)]


SYMBOLS = ("dq_context_create", "dq_context_destroy", "dq_problem_create", "dq_problem_set_vectors",
           "dq_problem_constants", "dq_problem_destroy", "dq_solve", "dq_solve_many", "dq_serve_start",
           "dq_submit", "dq_poll", "dq_serve_stop", "dq_context_profile", "dq_context_stats",
           "dq_autotune", "dq_solve_noalloc", "dq_test_tc_gemm", "dq_test_bounded_wait", "dq_theory",
           "dq_solve_theory", "dq_problem_create_sparse", "dq_last_error", "dq_version")

_lib = None


class DuquadError(RuntimeError):
    def __init__(self, status, msg):
        super().__init__(f"duquad status {status}: {msg}")
        self.status = status


def lib(build_if_needed: bool = True):
    """Load libduquad.so (building it in-tree when sources changed)."""
    global _lib
    if _lib is not None:
        return _lib
    path = _build.LIB
    if build_if_needed and not _build.up_to_date():
        _build.build()
    if not os.path.exists(path):
        raise ImportError(f"libduquad.so is missing at {path}; run paper_1504_05708_gb300._build.build()")
    L = ctypes.CDLL(path)
    P = ctypes.POINTER
    vp = ctypes.c_void_p
    st = ctypes.c_int
    L.dq_context_create.argtypes = [ctypes.c_int, vp, P(vp)]
    L.dq_context_destroy.argtypes = [vp]
    L.dq_problem_create.argtypes = [vp, P(ProblemDesc), P(vp)]
    L.dq_problem_set_vectors.argtypes = [vp, vp, vp, ctypes.c_int32]
    L.dq_problem_constants.argtypes = [vp, P(ctypes.c_double), P(ctypes.c_double), P(ctypes.c_double)]
    L.dq_problem_destroy.argtypes = [vp]
    L.dq_solve.argtypes = [vp, P(SolveOpts), P(Outputs), P(Result)]
    L.dq_solve_many.argtypes = [P(vp), ctypes.c_int32, P(SolveOpts), P(Outputs), P(Result)]
    L.dq_serve_start.argtypes = [vp, ctypes.c_int32, ctypes.c_int64]
    L.dq_submit.argtypes = [vp, vp, P(SolveOpts), vp, vp, P(ctypes.c_uint64)]
    L.dq_poll.argtypes = [vp, ctypes.c_uint64, vp, vp, vp, P(Result)]
    L.dq_serve_stop.argtypes = [vp]
    L.dq_test_tc_gemm.argtypes = [vp, vp, vp, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32, ctypes.c_int32,
                                  ctypes.c_int32, vp]
    L.dq_test_bounded_wait.argtypes = [ctypes.c_uint64, ctypes.c_int32, vp]
    L.dq_autotune.argtypes = [P(vp), ctypes.c_int32, P(SolveOpts), ctypes.c_int32, P(ctypes.c_int32),
                              P(ctypes.c_int32)]
    L.dq_solve_noalloc.argtypes = [ctypes.c_int, P(ProblemDesc), P(SolveOpts), P(Outputs), P(Result), vp]
    L.dq_context_profile.argtypes = [vp, ctypes.c_int32]
    L.dq_context_stats.argtypes = [vp, P(Stats), ctypes.c_int32]
    L.dq_theory.argtypes = [P(TheoryIn), P(TheoryOut)]
    L.dq_problem_create_sparse.argtypes = [vp, P(SparseDesc), P(vp)]
    L.dq_solve_theory.argtypes = [vp, P(TheorySolveOpts), P(Outputs), P(Result), P(TheoryOut),
                                  P(ctypes.c_double)]
    for name in SYMBOLS[:-2]:
        getattr(L, name).restype = st
    L.dq_last_error.restype = ctypes.c_char_p
    L.dq_version.restype = ctypes.c_char_p
    _lib = L
    return L


def theory(alg, eps, Rd, D_U, lmax_Q, lmin_Q, normG2, rho=NAN) -> dict:
    """Iteration counts of the theory mode (dq_theory): rho, LL, sigma, Ld, eps_in, k_out, k_in, k_total."""
    ti = TheoryIn(ALGS[alg] if isinstance(alg, str) else int(alg), eps, Rd, D_U, lmax_Q, lmin_Q, normG2, rho)
    to = TheoryOut()
    check(lib().dq_theory(ctypes.byref(ti), ctypes.byref(to)), (OK,))
    return {f: getattr(to, f) for f, _ in TheoryOut._fields_}


def check(status, allow=(OK, NOT_CONVERGED)):
    if status in allow:
        return status
    raise DuquadError(status, lib().dq_last_error().decode())


def _ptr(a):
    """Host numpy (double, C-contiguous) or torch tensor -> (pointer, keepalive)."""
    if a is None:
        return None, None
    if hasattr(a, "data_ptr"):
        if not a.is_contiguous():
            raise ValueError("tensor must be contiguous")
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=np.float64)
    return arr.ctypes.data, arr


def opts(alg="DFGM", *, output=OUT_BOTH, inner_stop=INNER_GAP, engine=ENGINE_AUTO, eps_out=1e-3,
         eps_in=NAN, rho=NAN, fixed_outer=0, fixed_inner=0, max_outer=0, max_inner=0, check_every=0,
         inner_check_every=0, warm_start=0, kd_literal=0, Ld=NAN, LL=NAN, sigma=NAN,
         fresh_constants=0, inner_cert=CERT_AUTO, f_star=None) -> SolveOpts:
    o = SolveOpts()
    o.alg = ALGS[alg] if isinstance(alg, str) else int(alg)
    o.output, o.inner_stop, o.engine = output, inner_stop, engine
    o.eps_out, o.eps_in, o.rho = eps_out, eps_in, rho
    o.fixed_outer, o.fixed_inner, o.max_outer, o.max_inner = fixed_outer, fixed_inner, max_outer, max_inner
    o.check_every, o.inner_check_every, o.warm_start, o.kd_literal = check_every, inner_check_every, warm_start, kd_literal
    o.Ld, o.LL, o.sigma = Ld, LL, sigma
    o.fresh_constants = fresh_constants
    if f_star is not None:  # the paper's stop on |F(u) - F*| for a known F*
        o.stop_fstar, o.f_star = 1, float(f_star)
    o.inner_cert = inner_cert
    if fixed_inner and inner_stop == INNER_GAP:
        o.inner_stop = INNER_FIXED
    return o


class Context:
    def __init__(self, device: int = 0, stream=None):
        """stream: a torch.cuda.Stream, a raw cudaStream_t int, or None (current torch stream)."""
        L = lib()
        if stream is None:
            import torch
            stream = torch.cuda.current_stream(device).cuda_stream
        elif hasattr(stream, "cuda_stream"):
            stream = stream.cuda_stream
        h = ctypes.c_void_p()
        check(L.dq_context_create(device, ctypes.c_void_p(stream), ctypes.byref(h)), (OK,))
        self.h = h
        self.device = device

    # ---- serving (continuous batching)
    def serve_start(self, slots: int = 1024, hbm_budget_bytes: int = 64 << 30):
        check(lib().dq_serve_start(self.h, slots, hbm_budget_bytes), (OK,))

    def submit(self, prob: "Problem", o: SolveOpts, q=None, g=None) -> int:
        t = ctypes.c_uint64()
        pq, kq = _ptr(q)
        pg, kg = _ptr(g)
        check(lib().dq_submit(self.h, prob.h, ctypes.byref(o), pq, pg, ctypes.byref(t)), (OK,))
        return t.value

    def poll(self, ticket: int, n: int, p: int):
        """None while pending, else (status, x_last, x_avg, lam, Result)."""
        xl, xa, lm = np.zeros(n), np.zeros(n), np.zeros(max(p, 1))
        r = Result()
        st = lib().dq_poll(self.h, ticket, xl.ctypes.data, xa.ctypes.data, lm.ctypes.data, ctypes.byref(r))
        if st == PENDING:
            return None
        check(st)
        return st, xl, xa, lm[:p], r

    def serve_stop(self):
        check(lib().dq_serve_stop(self.h), (OK,))

    def profile(self, enable: bool = True):
        check(lib().dq_context_profile(self.h, int(enable)), (OK,))

    def stats(self, reset: bool = False) -> dict:
        s = Stats()
        check(lib().dq_context_stats(self.h, ctypes.byref(s), int(reset)), (OK,))
        return {f: getattr(s, f) for f, _ in Stats._fields_}

    def close(self):
        if self.h:
            lib().dq_context_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Problem:
    """A device-resident QP (eq. original_primal).  Host arrays: numpy (converted
    to double); device arrays: torch CUDA tensors of the precision's dtype."""

    def __init__(self, ctx: Context, Q, q, G, g, lb, ub, *, prec=FP32, batch=1, cone=CONE_INEQ,
                 lmax_Q=NAN, lmin_Q=NAN, normG2=NAN, lipschitz=LIP_LANCZOS):
        self.ctx = ctx
        dev = hasattr(Q, "data_ptr") and getattr(Q, "is_cuda", False)
        n = int(q.shape[-1])
        p = int(g.shape[-1]) if g is not None else 0
        d = ProblemDesc()
        d.n, d.p, d.batch, d.cone, d.prec = n, p, batch, cone, prec
        d.memory = DEVICE if dev else HOST
        keep = []
        for f, a in (("Q", Q), ("q", q), ("G", G), ("g", g), ("lb", lb), ("ub", ub)):
            ptr, k = _ptr(a)
            keep.append(k)
            setattr(d, f, ptr)
        d.lmax_Q, d.lmin_Q, d.normG2 = lmax_Q, lmin_Q, normG2
        d.lipschitz = lipschitz
        h = ctypes.c_void_p()
        check(lib().dq_problem_create(ctx.h, ctypes.byref(d), ctypes.byref(h)), (OK,))
        self.h = h
        self.n, self.p, self.batch, self.prec = n, p, batch, prec
        self._borrowed = (Q, G) if dev else None

    def set_vectors(self, q=None, g=None):
        dev = (q is not None and hasattr(q, "data_ptr")) or (g is not None and hasattr(g, "data_ptr"))
        pq, kq = _ptr(q)
        pg, kg = _ptr(g)
        check(lib().dq_problem_set_vectors(self.h, pq, pg, DEVICE if dev else HOST), (OK,))

    def constants(self):
        a, b, c = ctypes.c_double(), ctypes.c_double(), ctypes.c_double()
        check(lib().dq_problem_constants(self.h, ctypes.byref(a), ctypes.byref(b), ctypes.byref(c)), (OK,))
        return a.value, b.value, c.value

    def solve(self, o: SolveOpts | None = None, *, device_out=None, **kw):
        """Solve; returns (x_last, x_avg, lam, [Result]) as host double arrays (batch-shaped), or
        writes into device tensors device_out=(x_last, x_avg, lam) and returns the results."""
        o = o or opts(**kw)
        B = self.batch
        res = (Result * B)()
        out = Outputs()
        if device_out is not None:
            xl, xa, lm = device_out
            out.x_last = xl.data_ptr() if xl is not None else None
            out.x_avg = xa.data_ptr() if xa is not None else None
            out.lambda_ = lm.data_ptr() if lm is not None else None
            out.memory = DEVICE
            st = lib().dq_solve(self.h, ctypes.byref(o), ctypes.byref(out), res)
            check(st)
            return list(res)
        xl = np.zeros((B, self.n))
        xa = np.zeros((B, self.n))
        lm = np.zeros((B, max(self.p, 1)))
        out.x_last, out.x_avg, out.lambda_ = xl.ctypes.data, xa.ctypes.data, lm.ctypes.data
        out.memory = HOST
        st = lib().dq_solve(self.h, ctypes.byref(o), ctypes.byref(out), res)
        check(st)
        lm = lm[:, :self.p]
        if B == 1:
            return xl[0], xa[0], lm[0], [res[0]]
        return xl, xa, lm, list(res)

    def solve_theory(self, alg, eps, *, Rd=NAN, safety=NAN, rho=NAN, max_total=0, engine=ENGINE_AUTO):
        """dq_solve_theory: the fixed counts of the analysis (with an R_d estimate when Rd is NaN).
        Returns (x_last, x_avg, lam, Result, counts dict, R_d used)."""
        t = TheorySolveOpts(ALGS[alg] if isinstance(alg, str) else int(alg), eps, Rd, safety, rho, max_total,
                            engine)
        xl, xa, lm = np.zeros(self.n), np.zeros(self.n), np.zeros(max(self.p, 1))
        out = Outputs()
        out.x_last, out.x_avg, out.lambda_, out.memory = xl.ctypes.data, xa.ctypes.data, lm.ctypes.data, HOST
        r, to, rd = Result(), TheoryOut(), ctypes.c_double()
        check(lib().dq_solve_theory(self.h, ctypes.byref(t), ctypes.byref(out), ctypes.byref(r), ctypes.byref(to),
                                    ctypes.byref(rd)))
        return xl, xa, lm[:self.p], r, {f: getattr(to, f) for f, _ in TheoryOut._fields_}, rd.value

    def close(self):
        if getattr(self, "h", None):
            lib().dq_problem_destroy(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


def _iptr(a):
    """Host numpy (int32, C-contiguous) or torch int32 tensor -> (pointer, keepalive)."""
    if hasattr(a, "data_ptr"):
        return a.data_ptr(), a
    arr = np.ascontiguousarray(a, dtype=np.int32)
    return arr.ctypes.data, arr


class SparseProblem(Problem):
    """A sparse QP (dq_problem_create_sparse): Q (full symmetric) and G as CSR triples
    (rowptr, col, val).  Host: numpy (int32 indices, values converted to double); device:
    torch CUDA tensors (int32 indices, values of the precision's dtype)."""

    def __init__(self, ctx: Context, Qcsr, q, Gcsr, g, lb, ub, *, prec=FP32, cone=CONE_INEQ, lmax_Q=NAN,
                 lmin_Q=NAN, normG2=NAN, lipschitz=LIP_LANCZOS):
        self.ctx = ctx
        dev = hasattr(q, "data_ptr") and getattr(q, "is_cuda", False)
        n = int(q.shape[-1])
        p = int(g.shape[-1]) if g is not None else 0
        d = SparseDesc()
        d.n, d.p, d.cone, d.prec, d.memory = n, p, cone, prec, DEVICE if dev else HOST
        keep = []
        for name, (rp, ci, va) in (("Q", Qcsr), ("G", Gcsr if p else (None, None, None))):
            if rp is None:
                continue
            prp, k1 = _iptr(rp)
            pci, k2 = _iptr(ci)
            pva, k3 = _ptr(va)
            keep += [k1, k2, k3]
            setattr(d, name + "_rowptr", prp)
            setattr(d, name + "_col", pci)
            setattr(d, name + "_val", pva)
            setattr(d, "nnz_" + name, int(ci.shape[0]))
        for f, a in (("q", q), ("g", g), ("lb", lb), ("ub", ub)):
            ptr, k = _ptr(a)
            keep.append(k)
            setattr(d, f, ptr)
        d.lmax_Q, d.lmin_Q, d.normG2 = lmax_Q, lmin_Q, normG2
        d.lipschitz = lipschitz
        h = ctypes.c_void_p()
        check(lib().dq_problem_create_sparse(ctx.h, ctypes.byref(d), ctypes.byref(h)), (OK,))
        self.h = h
        self.n, self.p, self.batch, self.prec = n, p, 1, prec
        self._borrowed = None


def autotune(problems, o_list, sample=256):
    """dq_autotune: pick (threads, smem cap) for this mix; returns the choice."""
    cnt = len(problems)
    hs = (ctypes.c_void_p * cnt)(*[p.h.value for p in problems])
    os_ = (SolveOpts * cnt)(*o_list)
    t, s = ctypes.c_int32(), ctypes.c_int32()
    check(lib().dq_autotune(hs, cnt, os_, sample, ctypes.byref(t), ctypes.byref(s)), (OK,))
    return t.value, s.value


def solve_many(problems, o_list, *, device_outs=None):
    """One persistent launch over many problems (dq_solve_many).  Returns per-problem
    host outputs (x_last, x_avg, lam) and the results, unless device_outs is given."""
    cnt = len(problems)
    hs = (ctypes.c_void_p * cnt)(*[p.h.value for p in problems])
    os_ = (SolveOpts * cnt)(*o_list)
    total = sum(p.batch for p in problems)
    res = (Result * total)()
    outs = (Outputs * cnt)()
    host = []
    for i, p in enumerate(problems):
        if device_outs is not None:
            xl, xa, lm = device_outs[i]
            outs[i].x_last = xl.data_ptr() if xl is not None else None
            outs[i].x_avg = xa.data_ptr() if xa is not None else None
            outs[i].lambda_ = lm.data_ptr() if lm is not None else None
            outs[i].memory = DEVICE
        else:
            xl = np.zeros((p.batch, p.n))
            xa = np.zeros((p.batch, p.n))
            lm = np.zeros((p.batch, max(p.p, 1)))
            host.append((xl, xa, lm))
            outs[i].x_last, outs[i].x_avg, outs[i].lambda_ = xl.ctypes.data, xa.ctypes.data, lm.ctypes.data
            outs[i].memory = HOST
    check(lib().dq_solve_many(hs, cnt, os_, outs, res))
    if device_outs is not None:
        return list(res)
    return [(h[0], h[1], h[2][:, :p.p]) for h, p in zip(host, problems)], list(res)
