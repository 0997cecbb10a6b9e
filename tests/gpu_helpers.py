"""Helpers shared by the GPU tests: build library problems from generator instances
and run the oracle on the same data and constants."""
import math

import numpy as np

import oracle as O
import workloads as W

ALG_IDS = {"DGM": O.DGM, "DFGM": O.DFGM, "ADGM": O.ADGM, "ADFGM": O.ADFGM}


def rel(a, b):
    a, b = np.asarray(a, float), np.asarray(b, float)
    nb = np.linalg.norm(b)
    return np.linalg.norm(a - b) / (nb if nb > 0 else 1.0)


def oracle_qp(inst):
    return O.QP(inst.Q, inst.q, inst.G, inst.g, inst.lb, inst.ub)


def exact_constants(inst, alg):
    """Oracle constants (LAPACK eigenvalues) used by both sides in parity runs."""
    return O.constants(oracle_qp(inst), ALG_IDS[alg], lmin_Q=inst.lmin_Q)


def gpu_problem(ctx, inst, prec, **kw):
    from paper_1504_05708_gb300 import duquad as D
    return D.Problem(ctx, inst.Q, inst.q, inst.G if inst.p else None, inst.g if inst.p else None,
                     inst.lb, inst.ub, prec=prec, lmin_Q=inst.lmin_Q, **kw)


def gpu_opts_from(c, alg, **kw):
    from paper_1504_05708_gb300 import duquad as D
    return D.opts(alg, rho=c.rho, LL=c.LL, Ld=c.Ld, sigma=c.sigma, **kw)
