"""Seeded synthetic QP generators shared by the tests, the benchmark and the oracle.

This module only draws random data; it holds none of the solver's arithmetic.
The instances stand in for the paper's random QPs (Sec. 6 of arXiv 1504.05708
uses randomly generated QPs and no public dataset):

  single_dense      dense QP with Q = U diag(Lambda) U', U Haar-orthogonal,
                    Lambda ~ U[lmin, lmax]; q ~ N(0,1); G ~ N(0, 1/n);
                    g = -|N(0,1)| - 0.1 (x = 0 strictly feasible); box [-1, 1].
                    n=50, p=25, Lambda ~ U[1,100], seed 0 is the FP64 case.
  large_dense       Q = M'M/n + 0.01 I with M ~ N(0,1) n x n; q ~ N(0,1);
                    G ~ N(0,1/n); g = -|N(0,1)| - 0.1; box [-1,1];
                    n=20000, p=10000 is the large FP32 case.
  mpc_batch         condensed MPC: nx=12, nu=4, horizon N=25 (n=100, p=600),
                    A random with spectral radius 0.95, B ~ N(0,1), Qx=I, R=0.1I,
                    B instances differing only in x0 ~ N(0,I).
  uneven_batch      instances as single_dense with n ~ U{16..512}, p = n/2,
                    kappa(Q) ~ U[10, 1e4] (lambda_1 = 1, lambda_n = kappa),
                    algorithm uniform over DGM/DFGM/ADGM/ADFGM.
  served_stream     Poisson arrival times and request mix for the served case.

Every generator returns known eigenvalue bounds (lmin_Q) where the
construction fixes them, so both the oracle and the GPU path can be handed
the same constants.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np

ALGS = ("DGM", "DFGM", "ADGM", "ADFGM")


@dataclass
class Instance:
    Q: np.ndarray
    q: np.ndarray
    G: np.ndarray
    g: np.ndarray
    lb: np.ndarray
    ub: np.ndarray
    lmin_Q: float
    lmax_Q: float | None = None
    alg: str = "DFGM"
    meta: dict = field(default_factory=dict)

    @property
    def n(self):
        return self.q.shape[0]

    @property
    def p(self):
        return self.g.shape[0]


def haar(rng: np.random.Generator, n: int) -> np.ndarray:
    """Haar-distributed orthogonal matrix: QR of a Gaussian with sign correction."""
    Z = rng.standard_normal((n, n))
    Qm, R = np.linalg.qr(Z)
    return Qm * np.sign(np.diag(R))[None, :]


def single_dense(n=50, p=25, seed=0, lam_lo=1.0, lam_hi=100.0, g_scale=1.0, g_offset=0.1,
                 box=1.0, alg="DFGM", kappa=None) -> Instance:
    """Dense QP with a prescribed spectrum (see module docstring).

    kappa given: lambda_1 = 1, lambda_n = kappa, the rest U[1, kappa].
    g_scale < 1 makes constraints active more often (parity variants)."""
    rng = np.random.default_rng(seed)
    U = haar(rng, n)
    if kappa is None:
        lam = rng.uniform(lam_lo, lam_hi, n)
    else:
        lam = np.concatenate([[1.0, kappa], rng.uniform(1.0, kappa, max(n - 2, 0))])[:n]
    Q = (U * lam[None, :]) @ U.T
    Q = 0.5 * (Q + Q.T)
    q = rng.standard_normal(n)
    G = rng.standard_normal((p, n)) / np.sqrt(n)
    g = -np.abs(rng.standard_normal(p)) * g_scale - g_offset
    lb = -box * np.ones(n)
    ub = box * np.ones(n)
    return Instance(Q, q, G, g, lb, ub, float(lam.min()), float(lam.max()), alg,
                    {"kind": "single_dense", "seed": seed})


def large_dense(n=20000, p=10000, seed=1, device="cpu", dtype=None, equality=False):
    """Large dense QP, Q = M'M/n + 0.01 I (lambda_min(Q) >= 0.01 by construction).

    Built with torch so the full-size case can be drawn directly in device
    memory; returns a dict of torch tensors (Q, q, G, g, lb, ub) plus lmin_Q.
    equality=True: g = -G u0 with u0 ~ U[-1/2, 1/2]^n, so G u + g = 0 has a
    solution inside the box (K = {0})."""
    import torch

    dtype = dtype or torch.float32
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    work = torch.float64 if (device == "cpu" or n <= 4096) else torch.float32
    M = torch.randn(n, n, generator=gen, device=device, dtype=work)
    Q = (M.T @ M) / n
    del M
    Q.diagonal().add_(0.01)
    Q = 0.5 * (Q + Q.T)
    q = torch.randn(n, generator=gen, device=device, dtype=work)
    G = torch.randn(p, n, generator=gen, device=device, dtype=work) / (n ** 0.5)
    g = -torch.randn(p, generator=gen, device=device, dtype=work).abs() - 0.1
    if equality:
        u0 = torch.rand(n, generator=gen, device=device, dtype=work) - 0.5
        g = -(G @ u0)
    lb = -torch.ones(n, device=device, dtype=work)
    ub = torch.ones(n, device=device, dtype=work)
    out = {k: v.to(dtype).contiguous() for k, v in dict(Q=Q, q=q, G=G, g=g, lb=lb, ub=ub).items()}
    out["lmin_Q"] = 0.01
    return out


def mpc_matrices(nx=12, nu=4, N=25, seed=2, rho_A=0.95):
    """System matrices and condensing operators of the MPC case.

    Returns dict with A, B, Gamma (N*nx x N*nu), Phi (N*nx x nx), Qbar, Rbar."""
    rng = np.random.default_rng(seed)
    A0 = rng.standard_normal((nx, nx))
    A = rho_A * A0 / np.max(np.abs(np.linalg.eigvals(A0)))
    B = rng.standard_normal((nx, nu))
    Gamma = np.zeros((N * nx, N * nu))
    Phi = np.zeros((N * nx, nx))
    Ak = np.eye(nx)
    powers = [np.eye(nx)]
    for _ in range(N):
        Ak = A @ Ak
        powers.append(Ak)
    for k in range(1, N + 1):  # state x_k, k = 1..N
        Phi[(k - 1) * nx:k * nx] = powers[k]
        for j in range(k):     # input u_j, j = 0..k-1
            Gamma[(k - 1) * nx:k * nx, j * nu:(j + 1) * nu] = powers[k - 1 - j] @ B
    return dict(A=A, B=B, Gamma=Gamma, Phi=Phi, Qbar=np.eye(N * nx), Rbar=0.1 * np.eye(N * nu),
                nx=nx, nu=nu, N=N)


def mpc_batch(batch=16384, nx=12, nu=4, N=25, seed=2, x0_seed=None):
    """Condensed-MPC QPs sharing Q and G; q and g are affine in x0 ~ N(0, I).

    Q = Gamma' Qbar Gamma + Rbar, q = Gamma' Qbar (Phi x0 - x_ref),
    G = [Gamma; -Gamma], g = [Phi x0 - b; -Phi x0 - b], box |u| <= 1,
    b = 1.05 max over the batch of max_k ||A^k x0||_inf (u = 0 strictly feasible),
    x_ref = 2 b on state 1 and 0 elsewhere (so state bounds become active).
    Returns dict(Q (n,n), G (p,n), qs (B,n), gs (B,p), lb, ub, lmin_Q, x0s)."""
    m = mpc_matrices(nx, nu, N, seed)
    rng = np.random.default_rng(seed + 1000 if x0_seed is None else x0_seed)
    x0s = rng.standard_normal((batch, nx))
    Gam, Phi = m["Gamma"], m["Phi"]
    free = x0s @ Phi.T                      # (B, N*nx) free response
    b = 1.05 * np.abs(free).max()
    x_ref = np.zeros(N * nx)
    x_ref[0::nx] = 2.0 * b
    Q = Gam.T @ m["Qbar"] @ Gam + m["Rbar"]
    Q = 0.5 * (Q + Q.T)
    qs = (free - x_ref[None, :]) @ m["Qbar"] @ Gam
    G = np.vstack([Gam, -Gam])
    gs = np.hstack([free - b, -free - b])
    n = N * nu
    return dict(Q=Q, G=G, qs=qs, gs=gs, lb=-np.ones(n), ub=np.ones(n), lmin_Q=0.1, x0s=x0s, b=b)


def uneven_sizes(count=10000, seed=3, n_lo=16, n_hi=512):
    """Sizes, conditioning and algorithm of each uneven-batch instance."""
    rng = np.random.default_rng(seed)
    ns = rng.integers(n_lo, n_hi + 1, count)
    kappas = rng.uniform(10.0, 1e4, count)
    algs = rng.integers(0, 4, count)
    seeds = rng.integers(0, 2**31 - 1, count)
    return ns, kappas, algs, seeds


def uneven_instance(n, kappa, alg, seed) -> Instance:
    """One uneven-batch instance: as single_dense with p = n/2 and kappa(Q) = kappa."""
    inst = single_dense(n=int(n), p=int(n) // 2, seed=int(seed), kappa=float(kappa),
                        alg=ALGS[int(alg)])
    inst.meta.update(kind="uneven", kappa=float(kappa))
    return inst


def uneven_batch(count=10000, seed=3, n_lo=16, n_hi=512):
    """List of uneven-batch instances (CPU, FP64).  count=10000 is the full case."""
    ns, kappas, algs, seeds = uneven_sizes(count, seed, n_lo, n_hi)
    return [uneven_instance(n, k, a, s) for n, k, a, s in zip(ns, kappas, algs, seeds)]


def served_stream(rate=20000.0, duration=60.0, seed=4, mpc_fraction=0.05):
    """Poisson arrival times (s) and request kinds (0 = uneven-batch QP, 1 = MPC)."""
    rng = np.random.default_rng(seed)
    count = rng.poisson(rate * duration)
    gaps = rng.exponential(1.0 / rate, count)
    t = np.cumsum(gaps)
    t = t[t < duration]
    kinds = (rng.random(t.size) < mpc_fraction).astype(np.int32)
    picks = rng.integers(0, 2**31 - 1, t.size)
    return t, kinds, picks


def uneven_batch_device(count=10000, seed=3, n_lo=16, n_hi=512, device="cuda", dtype=None):
    """The uneven batch drawn directly in device memory (torch), for the full-size case.

    Same distribution as uneven_instance (Haar eigenvectors, lambda_1 = 1,
    lambda_n = kappa, the rest U[1, kappa]; G ~ N(0, 1/n); g = -|N(0,1)| - 0.1;
    box [-1, 1]) with sizes, kappas and algorithms from uneven_sizes, but a torch
    random stream, so its entries differ from the host instances.  Returns a
    list of dicts (n, p, alg, Q, q, G, g, lb, ub) of `dtype` tensors."""
    import torch

    dtype = dtype or torch.float32
    ns, kappas, algs, _ = uneven_sizes(count, seed, n_lo, n_hi)
    gen = torch.Generator(device=device)
    gen.manual_seed(seed)
    out = [None] * count
    f64 = dict(device=device, dtype=torch.float64)
    for n in sorted(set(int(v) for v in ns)):
        idx = [i for i in range(count) if int(ns[i]) == n]
        b, p = len(idx), n // 2
        Z = torch.randn(b, n, n, generator=gen, **f64)
        U, R = torch.linalg.qr(Z)
        U = U * torch.sign(torch.diagonal(R, dim1=-2, dim2=-1)).unsqueeze(-2)
        kap = torch.tensor([float(kappas[i]) for i in idx], **f64)
        lam = 1.0 + torch.rand(b, n, generator=gen, **f64) * (kap[:, None] - 1.0)
        lam[:, 0] = 1.0
        if n > 1:
            lam[:, 1] = kap
        Q = (U * lam[:, None, :]) @ U.transpose(-1, -2)
        Q = 0.5 * (Q + Q.transpose(-1, -2))
        q = torch.randn(b, n, generator=gen, **f64)
        G = torch.randn(b, p, n, generator=gen, **f64) / n ** 0.5
        g = -torch.randn(b, p, generator=gen, **f64).abs() - 0.1
        for k, i in enumerate(idx):
            out[i] = dict(n=n, p=p, alg=ALGS[int(algs[i])], Q=Q[k].to(dtype).contiguous(),
                          q=q[k].to(dtype).contiguous(), G=G[k].to(dtype).contiguous(),
                          g=g[k].to(dtype).contiguous(), lb=-torch.ones(n, device=device, dtype=dtype),
                          ub=torch.ones(n, device=device, dtype=dtype))
    return out


def equality_dense(n=300, p=100, seed=0, lam_lo=1.0, lam_hi=100.0, n_zero=0, box=1.0) -> Instance:
    """Dense QP with equality constraints (K = {0}), feasible by construction.

    Q = U diag(lam) U' with lam ~ U[lam_lo, lam_hi] and n_zero of them set to 0
    (Q singular, the paper's Q >= 0 case); G ~ N(0, 1/n); g = -G u0 with
    u0 ~ U[-box/2, box/2] inside the box [-box, box]; q ~ N(0, 1)."""
    rng = np.random.default_rng(seed)
    U = haar(rng, n)
    lam = rng.uniform(lam_lo, lam_hi, n)
    lam[:n_zero] = 0.0
    Q = (U * lam[None, :]) @ U.T
    Q = 0.5 * (Q + Q.T)
    q = rng.standard_normal(n)
    G = rng.standard_normal((p, n)) / np.sqrt(n)
    u0 = rng.uniform(-0.5 * box, 0.5 * box, n)
    g = -G @ u0
    lb = -box * np.ones(n)
    ub = box * np.ones(n)
    inst = Instance(Q, q, G, g, lb, ub, float(lam.min()), float(lam.max()), "ADFGM",
                    {"kind": "equality_dense", "seed": seed, "cone": 1})
    return inst


def hidden_top(n=200, p=80, seed=0, lam_lo=1.0, lam_hi=100.0, lam_top=200.0, s_top=3.0):
    """Dense QP whose Q and G' G have their top eigenvectors orthogonal to the all-ones vector.

    v = (1, -1, 0, ..., 0) / sqrt(2).  Q = P A P + lam_top v v' with P = I - v v' and
    A = U diag(Lambda) U', Lambda ~ U[lam_lo, lam_hi] (so Q v = lam_top v and the rest of the
    spectrum lies in [0, lam_hi]); G = W diag(s) V' with V orthogonal, V e_1 = v, s_1 = s_top and
    the other singular values ~ U[0.1, 1] (so ||G||^2 = s_top^2 along v).  q ~ N(0,1);
    g = -|N(0,1)| - 0.1; box [-1, 1].  On v-perp, Q acts as A compressed to that subspace, whose
    eigenvalues lie in [lam_lo, lam_hi] (Cauchy interlacing); lmin_Q is LAPACK's smallest
    eigenvalue less a 1e-9 relative margin, lmax_Q LAPACK's largest (lam_top)."""
    rng = np.random.default_rng(seed)
    v = np.zeros(n)
    v[0], v[1] = 1.0, -1.0
    v /= np.sqrt(2.0)
    U = haar(rng, n)
    A = (U * rng.uniform(lam_lo, lam_hi, n)[None, :]) @ U.T
    Pm = np.eye(n) - np.outer(v, v)
    Q = Pm @ A @ Pm + lam_top * np.outer(v, v)
    Q = 0.5 * (Q + Q.T)
    Vb, R = np.linalg.qr(np.column_stack([v, rng.standard_normal((n, n - 1))]))
    Vb = Vb * np.sign(np.diag(R))[None, :]      # first column is +v
    Wm = haar(rng, p) if p else np.zeros((0, 0))
    k = min(n, p)
    s = np.concatenate([[s_top], rng.uniform(0.1, 1.0, max(k - 1, 0))])[:k]
    G = (Wm[:, :k] * s[None, :]) @ Vb[:, :k].T if p else np.zeros((0, n))
    q = rng.standard_normal(n)
    g = -np.abs(rng.standard_normal(p)) - 0.1
    ev = np.linalg.eigvalsh(Q)
    return Instance(Q, q, G, g, -np.ones(n), np.ones(n), float(ev[0]) * (1 - 1e-9), float(ev[-1]), "ADFGM",
                    {"kind": "hidden_top", "seed": seed})


def sparse_qp(n=100000, p=50000, deg=8, row_nnz=8, seed=6, dense=False):
    """Sparse QP in CSR form (the sparse case of Sec. 5, e.g. network utility maximisation).

    Q = L + diag(d): L the Laplacian of a random graph with about n deg / 2 edges (each node
    draws deg / 2 neighbours uniformly; weights ~ U[0.5, 1.5], repeated edges summed) and
    d ~ U[1, 10], so Q is symmetric with lambda_min(Q) >= 1 (L is PSD) and about (deg + 1) n
    nonzeros.  G is p x n with row_nnz distinct uniform columns per row, values N(0, 1/row_nnz);
    q ~ N(0,1); g = -|N(0,1)| - 0.1 (x = 0 strictly feasible); box [-1, 1].
    Returns a dict of numpy arrays: Q_rowptr, Q_col, Q_val, G_rowptr, G_col, G_val (int32
    indices, float64 values), q, g, lb, ub, lmin_Q = 1.0; dense=True adds Q and G as dense
    arrays (small n only)."""
    rng = np.random.default_rng(seed)
    half = max(deg // 2, 1)
    src = np.repeat(np.arange(n, dtype=np.int64), half)
    dst = rng.integers(0, n, src.size)
    keep = src != dst
    i, j = np.minimum(src[keep], dst[keep]), np.maximum(src[keep], dst[keep])
    w = rng.uniform(0.5, 1.5, i.size)
    key = i * n + j
    uk, inv = np.unique(key, return_inverse=True)
    wu = np.bincount(inv, weights=w)
    ei, ej = uk // n, uk % n
    d = rng.uniform(1.0, 10.0, n)
    diag = d + np.bincount(ei, weights=wu, minlength=n) + np.bincount(ej, weights=wu, minlength=n)
    rows = np.concatenate([np.arange(n), ei, ej])
    cols = np.concatenate([np.arange(n), ej, ei])
    vals = np.concatenate([diag, -wu, -wu])
    order = np.lexsort((cols, rows))
    rows, cols, vals = rows[order], cols[order], vals[order]
    Q_rowptr = np.zeros(n + 1, np.int64)
    np.add.at(Q_rowptr, rows + 1, 1)
    Q_rowptr = np.cumsum(Q_rowptr).astype(np.int32)
    # G: row_nnz distinct columns per row (sorted)
    k = min(row_nnz, n)
    G_col = _distinct_cols(rng, p, n, k).reshape(-1).astype(np.int32)
    G_val = rng.standard_normal(p * k) / np.sqrt(k)
    G_rowptr = (np.arange(p + 1) * k).astype(np.int32)
    q = rng.standard_normal(n)
    g = -np.abs(rng.standard_normal(p)) - 0.1
    out = dict(n=n, p=p, Q_rowptr=Q_rowptr, Q_col=cols.astype(np.int32), Q_val=vals, G_rowptr=G_rowptr,
               G_col=G_col, G_val=G_val, q=q, g=g, lb=-np.ones(n), ub=np.ones(n), lmin_Q=1.0)
    if dense:
        Q = np.zeros((n, n))
        Q[rows, cols] = vals
        G = np.zeros((p, n))
        G[np.repeat(np.arange(p), k), G_col] = G_val
        out["Q"], out["G"] = Q, G
    return out


def _distinct_cols(rng, p, n, k):
    """p rows of k distinct column indices in [0, n) (rejection of repeats, row by row)."""
    c = rng.integers(0, n, (p, k))
    for _ in range(64):
        s = np.sort(c, axis=1)
        dup = np.zeros_like(c, dtype=bool)
        dup[:, 1:] = s[:, 1:] == s[:, :-1]
        if not dup.any():
            return s
        s[dup] = rng.integers(0, n, int(dup.sum()))
        c = s
    raise RuntimeError("could not draw distinct columns")
