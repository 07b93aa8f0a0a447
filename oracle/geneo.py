"""H_k-GenEO local eigenproblems and the coarse space (oracle, FP64).

Def. (Eq. 5.12): on each overlapping subdomain Omega_i find p in V~_i (all
dofs of ovdof(Omega_i)) and lambda with
    b_{Omega_i}(p, v) = lambda (Xi_i p, Xi_i v)_{1,k,Omega_i}   for all v.
In matrices on ovdof(Omega_i): B^N p = lambda C p with
    B^N = local Neumann Helmholtz matrix  sum_{T in Omega_i} (K_T - k^2 M_T),
    C   = Xi D^N Xi,  D^N = sum_{T in Omega_i} (K_T + k^2 M_T),  Xi = diag(1/mu on dof, 0 else).
The lemma on indefinite pencils (Sec. 2.2) shows the finite eigenvalues are
real and the eigenvectors can be normalised c(p_l, p_m) = delta_lm.

Computation (exact in exact arithmetic): C vanishes on G = ovdof \\ dof, so
the G rows read B^N_GI p_I + B^N_GG p_G = 0.  Eliminating p_G leaves the
symmetric-definite pencil
    S p_I = lambda C_II p_I,   S = B^N_II - B^N_IG (B^N_GG)^{-1} B^N_GI,
whose eigenpairs are the finite eigenpairs of (B^N, C); the G directions are
the infinite ones.  scipy's symmetric-definite solver returns C_II-orthonormal
eigenvectors, which is the normalisation above.

Def. 5.1: keep the m_i smallest eigenvalues, with lambda_{m_i+1} > 0; the
coarse space is spanned by E_i Xi_i p_l, l <= m_i.  The numeric threshold
is a parameter tau > 0 (keep lambda < tau).  Eigenvalues tied across tau
(gap <= 1e-8 max(1, |tau|)) are kept together so that a degenerate
eigenspace is never split.  Because Xi_i is zero off dof(Omega_i), the
coarse vector is supported on dof(Omega_i) with values p_l / mu_l there.

The coarse operator B_0 = R_0 B E_0 (Eq. 2.23) is taken in its Galerkin
matrix form E = Z^T B Z with Z = [E_i Xi_i p_l] (Prop. 2.6 uses T_0 =
B_0^{-1} R_0 B in this form).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.linalg as sla
import scipy.sparse as sp

from .fem import assemble
from .decomposition import Subdomain, pou_weights


class EigenFailure(RuntimeError):
    pass


def local_pencil(xyz, elems, coeff, is_boundary, k, sd: Subdomain, mu):
    """(B^N, C) on ovdof(Omega_i), rows/cols in increasing global dof order."""
    A_loc, S_loc = assemble(xyz, elems, coeff, is_boundary, elem_subset=sd.elems)
    O = sd.ovdof
    BN = (A_loc - k * k * S_loc)[O][:, O].toarray()
    DN = (A_loc + k * k * S_loc)[O][:, O].toarray()
    w = pou_weights(sd, mu)
    C = w[:, None] * DN * w[None, :]
    return BN, C, w


def select_count(lam: np.ndarray, tau: float, cluster_tol: float = 1e-8) -> int:
    """Def. 5.1 with threshold tau: m = #{lambda < tau}, extended across ties."""
    m = int(np.count_nonzero(lam < tau))
    thr = cluster_tol * max(1.0, abs(tau))
    while 0 < m < lam.size and lam[m] - lam[m - 1] <= thr:
        m += 1
    return m


@dataclass
class LocalEigen:
    lam: np.ndarray       # all finite eigenvalues, ascending
    P: np.ndarray         # (|dof|, |dof|) C_II-orthonormal eigenvectors (columns)
    m: int                # kept count
    w_dof: np.ndarray     # 1/mu on dof(Omega_i)

    @property
    def Z(self) -> np.ndarray:
        """Coarse vectors on dof(Omega_i): Xi_i p_l = p_l / mu (Def. 5.1)."""
        return self.w_dof[:, None] * self.P[:, : self.m]


def reduced_pencil(BN, C, w):
    """(S, C_II) of the elimination described in the module docstring."""
    I = w > 0
    G = ~I
    BGG = BN[np.ix_(G, G)]
    if G.any():
        try:
            cf = sla.cho_factor(BGG)
        except np.linalg.LinAlgError as e:
            raise EigenFailure("B^N on ovdof minus dof is not positive definite") from e
        S = BN[np.ix_(I, I)] - BN[np.ix_(I, G)] @ sla.cho_solve(cf, BN[np.ix_(G, I)])
    else:
        S = BN[np.ix_(I, I)].copy()
    S = 0.5 * (S + S.T)
    return S, C[np.ix_(I, I)]


def local_eigen(BN, C, w, tau, cluster_tol: float = 1e-8) -> LocalEigen:
    S, CII = reduced_pencil(BN, C, w)
    lam, P = sla.eigh(S, CII)
    m = select_count(lam, tau, cluster_tol)
    return LocalEigen(lam, P, m, w[w > 0])


def finite_eigenvalues_qz(BN, C):
    """Independent route for small pencils: QZ on (B^N, C) directly, keeping
    the finite eigenvalues (|beta| not tiny)."""
    alpha, beta = sla.eig(BN, C, right=False, homogeneous_eigvals=True)
    scale = np.maximum(np.abs(alpha), np.abs(beta))
    fin = np.abs(beta) > 1e-10 * scale
    return np.sort((alpha[fin] / beta[fin]).real)


def coarse_basis(subs, eigs, n):
    """Z (n x n0, sparse): columns E_i Xi_i p_l stacked subdomain by subdomain."""
    rows, cols, vals = [], [], []
    c0 = 0
    for sd, ev in zip(subs, eigs):
        Zi = ev.Z
        r, c = np.meshgrid(sd.dof, np.arange(ev.m) + c0, indexing="ij")
        rows.append(r.ravel()); cols.append(c.ravel()); vals.append(Zi.ravel())
        c0 += ev.m
    if c0 == 0:
        return sp.csr_matrix((n, 0))
    return sp.csr_matrix((np.concatenate(vals), (np.concatenate(rows), np.concatenate(cols))), shape=(n, c0))


def coarse_matrix(B, Z) -> np.ndarray:
    """E = Z^T B Z (dense n0 x n0), the matrix of B_0 in Eq. 2.23."""
    return np.asarray((Z.T @ (B @ Z)).todense()) if Z.shape[1] else np.zeros((0, 0))
