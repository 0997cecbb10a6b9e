"""FP64 CPU oracle of DuQuad's inexact (augmented) dual first-order method.

TEST INFRASTRUCTURE ONLY.  Only ``tests/``, ``__graft_entry__.smoke()`` and the
CPU-baseline leg of ``bench.py`` may import this package.  The product path
(the CUDA library and its binding) never imports, links or calls it, and it
imports nothing from the product package.

The arithmetic lives in ``duquad_oracle.c`` (plain C, FP64, one loop per
formula of the paper); this module compiles it with gcc on first use and
wraps it with ctypes + numpy.  Citations (arXiv 1504.05708):
  * problem, Lagrangian, dual gradient: Sec. 2, eq. original_primal, auglag1, Ld
  * inner solver: Algorithm FOM and the GM / FGM / FGM_sigma rules, Sec. 2.1
  * outer solver: Algorithm DFOM, DGM / DFGM rules, Sec. 3
  * primal outputs: eq. last_primal and eq. average_primal, Sec. 4
``kkt.py`` holds an independent brute-force KKT enumeration used to pin it.
"""
from __future__ import annotations

import ctypes
import math
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "duquad_oracle.c")
_SO = os.path.join(_HERE, "_build", "libduquad_oracle.so")
_lock = threading.Lock()
_lib = None

DGM, DFGM, ADGM, ADFGM = 0, 1, 2, 3
ALG_NAMES = {"DGM": DGM, "DFGM": DFGM, "ADGM": ADGM, "ADFGM": ADFGM}
INNER_AUTO, INNER_GM, INNER_FGM, INNER_FGMSIGMA = 0, 1, 2, 3
CONE_INEQ, CONE_EQ = 0, 1
TRACE_COLS = 12
TRACE_FIELDS = ("k", "theta", "S", "beta", "inner", "dbar", "dg_dot_mu", "F", "dg_sq",
                "min_lambda", "norm_lambda", "infeas")


def build(force: bool = False) -> str:
    """Compile the oracle with gcc (-O2, no fast-math) into oracle/_build/."""
    os.makedirs(os.path.dirname(_SO), exist_ok=True)
    if force or not os.path.exists(_SO) or os.path.getmtime(_SO) < os.path.getmtime(_SRC):
        tmp = _SO + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c99", "-fPIC", "-shared", "-ffp-contract=off",
                               _SRC, "-o", tmp, "-lm"])
        os.replace(tmp, _SO)
    return _SO


class _QP(ctypes.Structure):
    _fields_ = [("n", ctypes.c_int), ("p", ctypes.c_int), ("cone", ctypes.c_int)] + [
        (f, ctypes.POINTER(ctypes.c_double)) for f in ("Q", "q", "G", "g", "lb", "ub")]


class _Opts(ctypes.Structure):
    _fields_ = [("alg", ctypes.c_int), ("rho", ctypes.c_double), ("LL", ctypes.c_double),
                ("sigma", ctypes.c_double), ("Ld", ctypes.c_double), ("kd_literal", ctypes.c_int),
                ("inner_variant", ctypes.c_int), ("inner_fixed", ctypes.c_int),
                ("eps_in", ctypes.c_double), ("inner_check_every", ctypes.c_int),
                ("max_inner", ctypes.c_int), ("outer_fixed", ctypes.c_int),
                ("eps_out", ctypes.c_double), ("outer_check_every", ctypes.c_int),
                ("max_outer", ctypes.c_int), ("want_last", ctypes.c_int),
                ("want_avg", ctypes.c_int), ("inner_cert_step", ctypes.c_int),
                ("stop_fstar", ctypes.c_int), ("f_star", ctypes.c_double)]


class _Res(ctypes.Structure):
    _fields_ = [("status", ctypes.c_int), ("outer_iters", ctypes.c_int),
                ("inner_iters", ctypes.c_longlong), ("converged_last", ctypes.c_int),
                ("converged_avg", ctypes.c_int), ("f_last", ctypes.c_double),
                ("infeas_last", ctypes.c_double), ("f_avg", ctypes.c_double),
                ("infeas_avg", ctypes.c_double), ("d_lb", ctypes.c_double)]


def _load():
    global _lib
    with _lock:
        if _lib is None:
            lib = ctypes.CDLL(build())
            P = ctypes.POINTER
            d = ctypes.c_double
            dp = P(d)
            qpp = P(_QP)
            lib.orc_F.restype = d
            lib.orc_F.argtypes = [qpp, dp]
            lib.orc_infeas.restype = d
            lib.orc_infeas.argtypes = [qpp, dp]
            lib.orc_lagrangian.restype = d
            lib.orc_lagrangian.argtypes = [qpp, d, dp, dp]
            lib.orc_dual_grad.restype = None
            lib.orc_dual_grad.argtypes = [qpp, d, dp, dp, dp]
            lib.orc_grad_lagr.restype = None
            lib.orc_grad_lagr.argtypes = [qpp, d, dp, dp, dp]
            lib.orc_fw_gap.restype = d
            lib.orc_fw_gap.argtypes = [qpp, d, dp, dp]
            lib.orc_inner_cert.restype = d
            lib.orc_inner_cert.argtypes = [qpp, d, dp, dp, d, d]
            lib.orc_fom.restype = ctypes.c_int
            lib.orc_step_cert.restype = d
            lib.orc_step_cert.argtypes = [qpp, d, dp, dp, d, d, dp]
            lib.orc_fom.argtypes = [qpp, d, dp, d, d, ctypes.c_int, ctypes.c_int, d, ctypes.c_int,
                                    ctypes.c_int, ctypes.c_int, dp, dp, ctypes.c_int]
            lib.orc_dfom.restype = ctypes.c_int
            lib.orc_dfom.argtypes = [qpp, P(_Opts), dp, dp, dp, dp, dp, P(_Res), dp, ctypes.c_int]
            lib.orc_power_lmax.restype = d
            lib.orc_power_lmax.argtypes = [qpp, ctypes.c_int, ctypes.c_int]
            _lib = lib
    return _lib


def _dp(a):
    return a.ctypes.data_as(ctypes.POINTER(ctypes.c_double)) if a is not None else None


def _f64(a):
    return None if a is None else np.ascontiguousarray(a, dtype=np.float64)


@dataclass
class QP:
    """A QP of eq. original_primal: Q (n,n) symmetric PSD, G (p,n), box [lb, ub]."""
    Q: np.ndarray
    q: np.ndarray
    G: np.ndarray
    g: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    cone: int = CONE_INEQ

    def __post_init__(self):
        self.Q, self.q, self.lb, self.ub = map(_f64, (self.Q, self.q, self.lb, self.ub))
        n = self.q.shape[0]
        self.G = _f64(self.G).reshape(-1, n)
        self.g = _f64(self.g).reshape(-1)

    @property
    def n(self):
        return self.q.shape[0]

    @property
    def p(self):
        return self.g.shape[0]

    def _c(self):
        s = _QP()
        s.n, s.p, s.cone = self.n, self.p, self.cone
        dummy = np.zeros(1)
        self._keep = (dummy,)
        s.Q, s.q, s.lb, s.ub = _dp(self.Q), _dp(self.q), _dp(self.lb), _dp(self.ub)
        s.G = _dp(self.G) if self.p else _dp(dummy)
        s.g = _dp(self.g) if self.p else _dp(dummy)
        return s


# ------------------------------------------------------------------ functions

def F(qp: QP, u) -> float:
    return _load().orc_F(ctypes.byref(qp._c()), _dp(_f64(u)))


def infeas(qp: QP, u) -> float:
    return _load().orc_infeas(ctypes.byref(qp._c()), _dp(_f64(u)))


def lagrangian(qp: QP, rho: float, u, lam) -> float:
    lam = _f64(lam) if qp.p else np.zeros(1)
    return _load().orc_lagrangian(ctypes.byref(qp._c()), rho, _dp(_f64(u)), _dp(lam))


def dual_grad(qp: QP, rho: float, u, lam) -> np.ndarray:
    out = np.zeros(max(qp.p, 1))
    lam = _f64(lam) if qp.p else np.zeros(1)
    _load().orc_dual_grad(ctypes.byref(qp._c()), rho, _dp(_f64(u)), _dp(lam), _dp(out))
    return out[:qp.p]


def grad_lagr(qp: QP, rho: float, u, lam) -> np.ndarray:
    out = np.zeros(qp.n)
    lam = _f64(lam) if qp.p else np.zeros(1)
    _load().orc_grad_lagr(ctypes.byref(qp._c()), rho, _dp(_f64(u)), _dp(lam), _dp(out))
    return out


def fw_gap(qp: QP, rho: float, x, lam) -> float:
    lam = _f64(lam) if qp.p else np.zeros(1)
    return _load().orc_fw_gap(ctypes.byref(qp._c()), rho, _dp(_f64(x)), _dp(lam))


def inner_cert(qp: QP, rho: float, x, lam, LL: float, sigma: float) -> float:
    """Upper bound on L_rho(x, lam) - d_rho(lam) used by the inner stopping rule (eq. duquad_in)."""
    lam = _f64(lam) if qp.p else np.zeros(1)
    return _load().orc_inner_cert(ctypes.byref(qp._c()), rho, _dp(_f64(x)), _dp(lam), LL, sigma)


def step_cert(qp: QP, rho: float, y, lam, LL: float, sigma: float):
    """Bound on L_rho(x+, lam) - d_rho(lam) for x+ = [y - grad/L]_U from any step point y
    (sigma > 0). Returns (bound, x+)."""
    lam = _f64(lam) if qp.p else np.zeros(1)
    xp = np.zeros(qp.n)
    b = _load().orc_step_cert(ctypes.byref(qp._c()), rho, _dp(_f64(y)), _dp(lam), LL, sigma, _dp(xp))
    return b, xp


def fom(qp: QP, rho, mu, LL, sigma, x0, *, variant=INNER_AUTO, fixed=0, eps_in=1e-8,
        check_every=1, max_inner=100000, phi_trace=0, cert_step=False):
    """Algorithm FOM on L_rho(., mu) over the box (Sec. 2.1). Returns (x, iters, phi[k]).
    cert_step: stop on the step certificate of y^k -> x^k (sigma > 0) instead of the
    certificate at x^k."""
    x = _f64(x0).copy()
    mu = _f64(mu) if qp.p else np.zeros(1)
    tr = np.zeros(max(phi_trace, 1))
    k = _load().orc_fom(ctypes.byref(qp._c()), rho, _dp(mu), LL, sigma, variant, fixed, eps_in,
                        check_every, max_inner, int(cert_step), _dp(x),
                        _dp(tr) if phi_trace else None, phi_trace)
    return x, k, tr[:min(k, phi_trace)] if phi_trace else None


def power_lmax(qp: QP, which: str = "Q", iters: int = 2000) -> float:
    """Rayleigh quotient of power iteration on Q ("Q") or G'G ("GtG")."""
    return _load().orc_power_lmax(ctypes.byref(qp._c()), 0 if which == "Q" else 1, iters)


# ------------------------------------------------------------------ constants

@dataclass
class Constants:
    """Step constants of Sec. 3: L_L = lmax(Q) + rho ||G||^2 (Step 1),
    sigma_L >= lmin(Q), L_d = ||G||^2 / (lmin(Q) + rho ||G||^2) (eq. Ld)."""
    rho: float
    LL: float
    sigma: float
    Ld: float
    lmax_Q: float
    lmin_Q: float
    normG2: float


def constants(qp: QP, alg: int, rho: float | None = None, lmin_Q: float | None = None,
              lmax_Q: float | None = None, normG2: float | None = None) -> Constants:
    """Exact constants via a dense symmetric eigen-solve (LAPACK, FP64).

    rho defaults to 0 for DGM/DFGM (Case 1) and 1/||G||^2 for ADGM/ADFGM."""
    ev = np.linalg.eigvalsh(qp.Q)
    lmax_Q = float(ev[-1]) if lmax_Q is None else float(lmax_Q)
    lmin_Q = max(float(ev[0]), 0.0) if lmin_Q is None else float(lmin_Q)
    if normG2 is None:
        normG2 = float(np.linalg.norm(qp.G, 2) ** 2) if qp.p else 0.0
    if rho is None:
        rho = 0.0 if alg in (DGM, DFGM) else (1.0 / normG2 if normG2 > 0 else 1.0)
    LL = lmax_Q + rho * normG2
    denom = lmin_Q + rho * normG2
    Ld = normG2 / denom if normG2 > 0 else 1.0
    return Constants(rho, LL, lmin_Q, Ld, lmax_Q, lmin_Q, normG2)


# ------------------------------------------------------------------ DFOM

@dataclass
class Result:
    x_last: np.ndarray
    x_avg: np.ndarray
    lam: np.ndarray
    status: int
    outer_iters: int
    inner_iters: int
    converged_last: bool
    converged_avg: bool
    f_last: float
    infeas_last: float
    f_avg: float
    infeas_avg: float
    d_lb: float
    trace: np.ndarray | None


def dfom(qp: QP, alg: int, c: Constants, *, inner_fixed=0, eps_in=1e-6, inner_check_every=1,
         max_inner=100000, outer_fixed=0, eps_out=1e-3, outer_check_every=1, max_outer=10000,
         want_last=True, want_avg=True, lambda0=None, x0=None, kd_literal=False,
         inner_variant=INNER_AUTO, trace_cap=0, inner_cert_step=False, f_star=None) -> Result:
    """Algorithm DFOM(d_rho, K_d) (Sec. 3) with both primal outputs (Sec. 4)."""
    o = _Opts()
    o.alg, o.rho, o.LL, o.sigma, o.Ld = alg, c.rho, c.LL, c.sigma, c.Ld
    o.kd_literal, o.inner_variant = int(kd_literal), inner_variant
    o.inner_fixed, o.eps_in, o.inner_check_every, o.max_inner = inner_fixed, eps_in, inner_check_every, max_inner
    o.outer_fixed, o.eps_out, o.outer_check_every, o.max_outer = outer_fixed, eps_out, outer_check_every, max_outer
    o.want_last, o.want_avg = int(want_last), int(want_avg)
    o.inner_cert_step = int(inner_cert_step)
    if f_star is not None:  # the paper's stop on |F(u) - F*| (Sec. 6) for a known F*
        o.stop_fstar, o.f_star = 1, float(f_star)
    n, p = qp.n, qp.p
    xl, xa, lam = np.zeros(n), np.zeros(n), np.zeros(max(p, 1))
    l0 = _f64(lambda0) if (lambda0 is not None and p) else None
    x0 = _f64(x0)
    cap = trace_cap
    tr = np.zeros(max(cap, 1) * TRACE_COLS)
    r = _Res()
    _load().orc_dfom(ctypes.byref(qp._c()), ctypes.byref(o), _dp(l0), _dp(x0), _dp(xl), _dp(xa),
                     _dp(lam), ctypes.byref(r), _dp(tr) if cap else None, cap)
    trace = None
    if cap:
        trace = tr.reshape(-1, TRACE_COLS)[:min(r.outer_iters, cap)]
    return Result(xl, xa, lam[:p], r.status, r.outer_iters, r.inner_iters, bool(r.converged_last),
                  bool(r.converged_avg), r.f_last, r.infeas_last, r.f_avg, r.infeas_avg, r.d_lb, trace)


def default_eps_in(alg: int, eps: float, Ld: float, Rd: float = 1.0) -> float:
    """Inner accuracy of eq. choose_ein: eps/4 for (A)DGM, eps^{3/2}/(8 R_d sqrt(2 L_d)) for (A)DFGM."""
    if alg in (DGM, ADGM):
        return eps / 4.0
    return eps * math.sqrt(eps) / (8.0 * Rd * math.sqrt(2.0 * Ld))


def k_out(alg: int, eps: float, Ld: float, Rd: float) -> float:
    """Outer iteration count of eq. choose_ein."""
    v = 8.0 * Ld * Rd * Rd / eps
    return v if alg in (DGM, ADGM) else math.sqrt(v)


def k_in(LL: float, sigma: float, D_U: float, eps_in: float) -> float:
    """Inner iteration count of Algorithm FOM for accuracy eps_in (Sec. 5, proof of the
    total-complexity theorem, from Lemma sublin_dfg with R_L = D_U):
    sqrt(2 L D_U^2 / eps_in) for sigma = 0, sqrt(L / sigma) log(L D_U^2 / eps_in) + 1 for sigma > 0."""
    if sigma > 0.0:
        return math.sqrt(LL / sigma) * math.log(LL * D_U * D_U / eps_in) + 1.0
    return math.sqrt(2.0 * LL * D_U * D_U / eps_in)


def rho_star(eps: float, Rd: float) -> float:
    """The smoothing that minimises k_out k_in (Sec. 5): rho* = 8 R_d^2 / eps."""
    return 8.0 * Rd * Rd / eps


from .sampled import sampled_fom_step  # noqa: E402,F401
