"""Brute-force KKT enumeration for tiny QPs (test infrastructure only).

An independent route to the exact solution of eq. original_primal (Sec. 2,
arXiv 1504.05708) used to pin the DFOM oracle: it shares nothing with the
iterative method.  For every combination of (variable at lb / at ub / free) and
(constraint active / inactive) it solves the KKT equality system with LAPACK and
keeps the combination that satisfies all sign and feasibility conditions.
With Q positive definite the QP has a unique solution and exactly this
combination (up to degenerate ties) passes.
"""
from __future__ import annotations

import itertools

import numpy as np


def solve_kkt(Q, q, G, g, lb, ub, *, box_active=True, equality=False, tol=1e-9):
    """Return (x*, lambda*, F*) of min 1/2 x'Qx + q'x s.t. Gx + g <= 0 (or = 0), lb <= x <= ub.

    box_active=False enumerates only the linear constraints (use it when the box
    is known to be inactive at the solution, e.g. a very wide box); the result is
    then checked against the box.  Cost: 3^n * 2^p (or 2^p) dense solves.
    """
    Q = np.asarray(Q, float)
    q = np.asarray(q, float)
    G = np.asarray(G, float).reshape(-1, q.size)
    g = np.asarray(g, float).reshape(-1)
    lb = np.asarray(lb, float)
    ub = np.asarray(ub, float)
    n, p = q.size, g.size
    var_states = [(0, 1, 2)] * n if box_active else [(0,)] * n  # 0 free, 1 at lb, 2 at ub
    con_states = [(1,)] * p if equality else [(0, 1)] * p      # 1 active
    best = None
    for vs in itertools.product(*var_states):
        fixed = np.array([s != 0 for s in vs], bool)
        xfix = np.where(np.array(vs) == 1, lb, ub)
        free = np.where(~fixed)[0]
        for cs in itertools.product(*con_states):
            act = np.where(np.array(cs, int) == 1)[0] if p else np.zeros(0, int)
            nf, na = free.size, act.size
            # unknowns [x_free, lambda_act]
            K = np.zeros((nf + na, nf + na))
            rhs = np.zeros(nf + na)
            xf = np.where(fixed, xfix, 0.0)
            K[:nf, :nf] = Q[np.ix_(free, free)]
            K[:nf, nf:] = G[np.ix_(act, free)].T
            rhs[:nf] = -(q[free] + Q[np.ix_(free, np.where(fixed)[0])] @ xf[fixed])
            K[nf:, :nf] = G[np.ix_(act, free)]
            rhs[nf:] = -(g[act] + G[np.ix_(act, np.where(fixed)[0])] @ xf[fixed])
            if nf + na:
                try:
                    sol = np.linalg.solve(K, rhs)
                except np.linalg.LinAlgError:
                    continue
                if not np.all(np.isfinite(sol)):
                    continue
            else:
                sol = np.zeros(0)
            x = xf.copy()
            x[free] = sol[:nf]
            lam = np.zeros(p)
            lam[act] = sol[nf:]
            # primal feasibility
            if np.any(x < lb - tol) or np.any(x > ub + tol):
                continue
            r = G @ x + g if p else np.zeros(0)
            if equality:
                if np.any(np.abs(r) > tol * max(1.0, np.abs(g).max(initial=0))):
                    continue
            else:
                if np.any(r > tol):
                    continue
                if np.any(lam < -tol):
                    continue
            # stationarity signs on the box
            grad = Q @ x + q + (G.T @ lam if p else 0.0)
            ok = True
            for i in range(n):
                if vs[i] == 1 and grad[i] < -tol:
                    ok = False
                if vs[i] == 2 and grad[i] > tol:
                    ok = False
                if vs[i] == 0 and abs(grad[i]) > 1e-7 * max(1.0, np.abs(q).max()):
                    ok = False
            if not ok:
                continue
            f = 0.5 * x @ Q @ x + q @ x
            if best is None or f < best[2]:
                best = (x, lam, f)
    if best is None:
        raise RuntimeError("no KKT point found (degenerate or infeasible instance)")
    return best
