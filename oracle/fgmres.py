"""Right-preconditioned flexible GMRES(m) (oracle, FP64).

The paper analyses GMRES on the preconditioned system of Eq. 2.24 (Thm. 3.1).
This solver applies the same preconditioner on the right, in flexible form
(the preconditioned directions z_j = M^{-1} v_j are stored), with the
Euclidean inner product, modified Gram-Schmidt Arnoldi and Givens rotations
(Saad, "Iterative Methods for Sparse Linear Systems", 2nd ed., Alg. 9.6).

Stopping: after each inner step j the recurrence residual |g_{j+1}| is
compared with tol * ||f||.  When it passes, when the cycle reaches `restart`
steps, on a happy breakdown, or at `max_iters`, the iterate is formed,
x += Z_j y with H_j y = g, and the true residual ||f - B x|| / ||f|| is
computed; the solve ends when that is <= tol (or at max_iters), otherwise a
new cycle starts from the true residual.  x_0 = 0.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class FGMRESResult:
    x: np.ndarray
    iters: int
    converged: bool
    true_rel_res: float
    history: list = field(default_factory=list)   # |g_{j+1}| / ||f|| per inner step


def fgmres(matvec, precond, f, tol=1e-8, restart=50, max_iters=1000) -> FGMRESResult:
    n = f.size
    x = np.zeros(n)
    nf = float(np.linalg.norm(f))
    if nf == 0.0:
        return FGMRESResult(x, 0, True, 0.0, [])
    hist = []
    iters = 0
    r = f.copy()
    true_rel = 1.0
    while True:
        beta = float(np.linalg.norm(r))
        m = restart
        V = np.zeros((m + 1, n))
        Zk = np.zeros((m, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        jd = 0
        for j in range(m):
            Zk[j] = precond(V[j])
            w = matvec(Zk[j])
            for i in range(j + 1):
                H[i, j] = float(np.dot(w, V[i]))
                w = w - H[i, j] * V[i]
            H[j + 1, j] = float(np.linalg.norm(w))
            breakdown = H[j + 1, j] == 0.0
            if not breakdown:
                V[j + 1] = w / H[j + 1, j]
            for i in range(j):
                t = cs[i] * H[i, j] + sn[i] * H[i + 1, j]
                H[i + 1, j] = -sn[i] * H[i, j] + cs[i] * H[i + 1, j]
                H[i, j] = t
            den = float(np.hypot(H[j, j], H[j + 1, j]))
            cs[j] = H[j, j] / den
            sn[j] = H[j + 1, j] / den
            H[j, j] = den
            H[j + 1, j] = 0.0
            g[j + 1] = -sn[j] * g[j]
            g[j] = cs[j] * g[j]
            iters += 1
            jd = j + 1
            hist.append(abs(g[j + 1]) / nf)
            if abs(g[j + 1]) <= tol * nf or iters >= max_iters or breakdown:
                break
        y = sla.solve_triangular(H[:jd, :jd], g[:jd], lower=False)
        x = x + Zk[:jd].T @ y
        r = f - matvec(x)
        true_rel = float(np.linalg.norm(r)) / nf
        if true_rel <= tol:
            return FGMRESResult(x, iters, True, true_rel, hist)
        if iters >= max_iters:
            return FGMRESResult(x, iters, False, true_rel, hist)
