"""One step of Algorithm FOM evaluated at selected coordinates (test infrastructure only).

Used to check the large-instance GPU path at full size, where a whole oracle
solve is out of reach: the step x+ = [y - grad_u L_rho(y, mu) / L]_U (Sec. 2.1,
step 1 of Algorithm FOM) needs the full G y (for w) but only the sampled rows
of Q and columns of G.  FP64 numpy; matrix products are library primitives.
"""
from __future__ import annotations

import numpy as np

CONE_INEQ, CONE_EQ = 0, 1


def sampled_fom_step(*, q, g, G, Q_rows, rows, y, mu, rho, L, lb, ub, Qy_full=None, cone=CONE_INEQ):
    """x+ at coordinates `rows` (all coordinates when rows is None, then Qy_full = Q y is given).

    grad_u L_rho(y, mu) = Q y + q + G' w with w = rho (z - [z]_K), z = G y + g + mu/rho for rho > 0
    and w = mu for rho = 0 (derivative of eq. auglag1)."""
    y = np.asarray(y, np.float64)
    Gy = G @ y
    if rho > 0:
        z = Gy + g + mu / rho
        zK = np.zeros_like(z) if cone == CONE_EQ else np.minimum(z, 0.0)
        w = rho * (z - zK)
    else:
        w = np.asarray(mu, np.float64)
    if rows is None:
        Qy = np.asarray(Qy_full, np.float64)
        Gtw = G.T @ w
        sel = slice(None)
    else:
        Qy = Q_rows @ y
        Gtw = G[:, rows].T @ w
        sel = rows
    grad = Qy + q[sel] + Gtw
    return np.clip(y[sel] - grad / L, lb[sel], ub[sel])
