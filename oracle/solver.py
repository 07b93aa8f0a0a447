"""Setup and solve pipeline of the oracle, mirroring the library boundary:
setup(mesh, coefficients, k, partition, overlap, tau) -> handle;
solve(handle, rhs, tol) -> u, iterations, residual history, true residual.

Setup follows the paper's order: Galerkin matrices (Sec. 2.1), overlapping
decomposition and partition of unity (Def. 2.3, 3.2, 2.7), local
eigenproblems (Eq. 5.12) and coarse space (Def. 5.1), preconditioner
(Eq. 2.22-2.23).  Solve is right-preconditioned FGMRES.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

from . import decomposition, fem, geneo, schwarz
from .fgmres import fgmres
from .gmres_dk import gmres_left_dk


@dataclass
class OracleHandle:
    B: object
    Dk: object
    subs: list
    mu: np.ndarray
    eigs: list
    Z: object
    precond: schwarz.AdditiveSchwarz
    restart: int
    max_iters: int
    Lambda: int

    @property
    def n(self) -> int:
        return self.B.shape[0]

    @property
    def m_i(self):
        return [e.m for e in self.eigs]

    @property
    def n0(self) -> int:
        return int(sum(self.m_i))

    def kept_eigenvalues(self):
        return [e.lam[: e.m] for e in self.eigs]


def setup(xyz, elems, is_boundary, coeff, k, elem_to_sub, n_sub, overlap=2, tau=0.5,
          levels="two", weighting="as", restart=50, max_iters=1000, nested=None) -> OracleHandle:
    """nested = (elem_to_fine, fine_overlap): the two decompositions of Sec. 2.3; the eigenproblems and the
    coarse space on the coarse subdomains, the local solves (Eq. 2.22) on the fine ones, Lambda over the
    fine ones.  The handle's subs and mu are then the fine ones; coarse_subs and mu_c the coarse ones."""
    B, Dk, _, _ = fem.helmholtz_matrices(xyz, elems, coeff, is_boundary, k)
    if nested is None:
        subs, mu = decomposition.decompose(xyz, elems, is_boundary, elem_to_sub, n_sub, overlap)
        csubs, mu_c = subs, mu
    else:
        csubs, mu_c, subs, _, mu = decomposition.decompose_nested(xyz, elems, is_boundary, elem_to_sub, n_sub,
                                                                  overlap, nested[0], nested[1])
    if mu_c.min() < 1 or mu.min() < 1:
        raise ValueError("some dof lies in no dof(Omega_i): the partition of unity is undefined")
    Lam = decomposition.multiplicity_lambda(elems, subs, elems.shape[0])
    eigs, Z = [], None
    if levels in ("two", "coarse"):
        for sd in csubs:
            BN, C, w = geneo.local_pencil(xyz, elems, coeff, is_boundary, k, sd, mu_c)
            eigs.append(geneo.local_eigen(BN, C, w, tau))
        Z = geneo.coarse_basis(csubs, eigs, B.shape[0])
    pc = schwarz.AdditiveSchwarz(B, subs, mu, Z, levels, weighting)
    h = OracleHandle(B, Dk, subs, mu, eigs, Z, pc, restart, max_iters, Lam)
    h.coarse_subs, h.mu_c = csubs, mu_c
    return h


def setup_problem(p, levels="two", weighting="as", nested=None) -> OracleHandle:
    """Convenience wrapper for a workloads.Problem-like object (nested: (elem_to_fine, fine_overlap))."""
    m = p.mesh
    return setup(m.xyz, m.elems, m.is_boundary, p.coeff, p.k, p.elem_to_sub, p.n_sub,
                 p.overlap, p.tau, levels, weighting, p.restart, p.max_iters, nested)


def load_vector(p) -> np.ndarray:
    """The problem's right-hand sides as load vectors, (n_rhs, n)."""
    if p.rhs is not None:
        return np.atleast_2d(p.rhs)
    m = p.mesh
    return fem.load_vector_nodal(m.xyz, m.elems, m.is_boundary, p.f_nodal)[None, :]


def solve(h: OracleHandle, rhs: np.ndarray, tol=1e-8):
    """Solves each right-hand side (rows of rhs) independently."""
    rhs = np.atleast_2d(rhs)
    out = []
    for f in rhs:
        out.append(fgmres(lambda v: h.B @ v, h.precond.apply, f, tol, h.restart, h.max_iters))
    return out


def solve_left_dk(h: OracleHandle, rhs: np.ndarray, tol=1e-8):
    """Left-preconditioned GMRES in the D_k inner product (the setting of Thm. 3.1) for each right-hand side."""
    rhs = np.atleast_2d(rhs)
    return [gmres_left_dk(lambda v: h.B @ v, h.precond.apply, h.Dk, f, tol, h.restart, h.max_iters) for f in rhs]
