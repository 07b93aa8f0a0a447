"""Left-preconditioned GMRES(m) in the D_k inner product, and the quantities of Thm. 3.1 (oracle, FP64).

TEST INFRASTRUCTURE ONLY (see the package docstring).

Thm. 3.1 bounds GMRES applied to the preconditioned system of Eq. 2.24, M^{-1} B u = M^{-1} f, when its
Arnoldi process and its residual minimisation use the inner product <x, y>_D = y^T D_k x, D_k = A + k^2 S
(Prop. 2.6, the matrix of the (.,.)_{1,k} inner product).  This is GMRES (Saad, "Iterative Methods for
Sparse Linear Systems", 2nd ed., Alg. 6.9, restarted) with every inner product and norm taken in that
inner product:
  r_0 = M^{-1} f (x_0 = 0), beta = ||r_0||_D, v_1 = r_0 / beta;
  step j: w = M^{-1} B v_j; h_ij = <w, v_i>_D for i = 1..j (modified Gram-Schmidt), w -= h_ij v_i;
          h_{j+1,j} = ||w||_D, v_{j+1} = w / h_{j+1,j};
  Givens rotations reduce H to triangular form; |g_{j+1}| is ||M^{-1}(f - B x_j)||_D for the minimiser
  x_j over x_0 + span(v_1..v_j).
Stopping: after each step, |g_{j+1}| <= tol * ||M^{-1} f||_D (the norm of Eq. 4.22, relative to the first
cycle's), or the cycle is full, or max_iters, or a happy breakdown; then x += V_j y (H_j y = g) and the
preconditioned residual M^{-1}(f - B x) is recomputed; the solve ends when its D_k norm is
<= tol * ||M^{-1} f||_D, otherwise a new cycle starts from it.
"""
from __future__ import annotations

from dataclasses import dataclass, field

import numpy as np
import scipy.linalg as sla


@dataclass
class DkGMRESResult:
    x: np.ndarray
    iters: int
    converged: bool
    pc_rel_res: float      # ||M^{-1}(f - B x)||_D / ||M^{-1} f||_D at the end
    true_rel_res: float    # ||f - B x|| / ||f|| at the end
    history: list = field(default_factory=list)  # |g_{j+1}| / ||M^{-1} f||_D per inner step


def gmres_left_dk(matvec, precond, D, f, tol=1e-8, restart=50, max_iters=1000) -> DkGMRESResult:
    """matvec(x) = B x, precond(v) = M^{-1} v, D: the D_k matrix (sparse or dense), f: load vector."""
    def dot(x, y):
        return float(y @ (D @ x))

    n = f.size
    x = np.zeros(n)
    nf = float(np.linalg.norm(f))
    if nf == 0.0:
        return DkGMRESResult(x, 0, True, 0.0, 0.0, [])
    r = precond(f)
    beta0 = np.sqrt(dot(r, r))
    hist = []
    iters = 0
    while True:
        beta = np.sqrt(dot(r, r))
        m = restart
        V = np.zeros((m + 1, n))
        H = np.zeros((m + 1, m))
        cs = np.zeros(m)
        sn = np.zeros(m)
        g = np.zeros(m + 1)
        g[0] = beta
        V[0] = r / beta
        jd = 0
        for j in range(m):
            w = precond(matvec(V[j]))
            for i in range(j + 1):
                H[i, j] = dot(w, V[i])
                w = w - H[i, j] * V[i]
            H[j + 1, j] = np.sqrt(dot(w, w))
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
            hist.append(abs(g[j + 1]) / beta0)
            if abs(g[j + 1]) <= tol * beta0 or iters >= max_iters or breakdown:
                break
        y = sla.solve_triangular(H[:jd, :jd], g[:jd], lower=False)
        x = x + V[:jd].T @ y
        r = precond(f - matvec(x))
        pc_rel = np.sqrt(dot(r, r)) / beta0
        if pc_rel <= tol or iters >= max_iters:
            true_rel = float(np.linalg.norm(f - matvec(x))) / nf
            return DkGMRESResult(x, iters, bool(pc_rel <= tol), float(pc_rel), true_rel, hist)


def tau_next(eigs) -> float:
    """tau of Thm. 3.1 (Def. 5.1 notation): min over subdomains of lambda_{m_i+1}, the smallest local
    eigenvalue left out of the coarse space (inf if every subdomain kept its whole spectrum)."""
    vals = [e.lam[e.m] for e in eigs if e.m < e.lam.size]
    return float(min(vals)) if vals else float("inf")


def theory(Lambda: float, tau: float, k: float, H_f: float, c_stab: float) -> dict:
    """Thm. 3.1: Theta = 1 / tau, s of Eq. 4.3 and gamma of Eq. 4.5 (the residual contraction
    (1 - gamma^2)^{1/2} per step of Eq. 4.22 is guaranteed when s < 1)."""
    Theta = 1.0 / tau
    a = 2.0 + 3.0 * Lambda ** 4 * Theta
    s = 2.0 * Lambda ** 2 * a * (2.0 * k * np.sqrt(Theta) * (1.0 + c_stab) + 3.0 * k * H_f)
    gamma = (1.0 - s) / (a * (18.0 + 8.0 * Lambda ** 3))
    return {"Lambda": Lambda, "tau": tau, "Theta": Theta, "s": s, "gamma": gamma, "guaranteed": s < 1.0}
