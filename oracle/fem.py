"""P1 finite-element matrices of the Helmholtz problem (oracle, FP64).

Sec. 2.1 of the paper: the Galerkin system B u = f (Eq. 2.11, 2.12) with
(B)_ij = b(phi_j, phi_i), b(u,v) = int A grad u . grad v - k^2 u v, and the
matrices A (stiffness, a(.,.)) and S (mass, (.,.)).  Prop. 2.6 introduces
D_k = A + k^2 S.  The coefficient A is the scalar a_T times the identity on
each element T.

Element matrices of a d-simplex T with barycentric gradients g_0..g_d:
  stiffness  K_T[i,j] = a_T |T| g_i . g_j
  mass       M_T[i,j] = |T| (1 + delta_ij) / ((d+1)(d+2))      (exact for P1)
"""
from __future__ import annotations

import math

import numpy as np
import scipy.sparse as sp


def barycentric_gradients(xyz: np.ndarray, elems: np.ndarray):
    """Per element: (|T|, gradients of the d+1 barycentric coordinates)."""
    d = xyz.shape[1]
    P = xyz[elems]                                  # (ne, d+1, d)
    Ed = np.transpose(P[:, 1:, :] - P[:, :1, :], (0, 2, 1))   # columns = edges x_i - x_0
    det = np.linalg.det(Ed)
    vol = np.abs(det) / math.factorial(d)
    Einv = np.linalg.inv(Ed)                        # rows i = grad of lambda_{i+1}
    g = np.concatenate([-Einv.sum(axis=1, keepdims=True), Einv], axis=1)   # (ne, d+1, d)
    return vol, g


def element_matrices(xyz: np.ndarray, elems: np.ndarray, coeff: np.ndarray):
    """Element stiffness (with a_T) and mass matrices, shape (ne, d+1, d+1)."""
    d = xyz.shape[1]
    vol, g = barycentric_gradients(xyz, elems)
    K = coeff[:, None, None] * vol[:, None, None] * np.einsum("eid,ejd->eij", g, g)
    base = (np.ones((d + 1, d + 1)) + np.eye(d + 1)) / ((d + 1) * (d + 2))
    M = vol[:, None, None] * base[None, :, :]
    return K, M


def dof_map(is_boundary: np.ndarray) -> np.ndarray:
    """Global dof of each node; -1 on Dirichlet nodes (V^h in H^1_0, Sec. 2.1)."""
    d = np.full(is_boundary.size, -1, dtype=np.int64)
    inner = np.flatnonzero(is_boundary == 0)
    d[inner] = np.arange(inner.size)
    return d


def assemble(xyz, elems, coeff, is_boundary, elem_subset=None):
    """Stiffness A and mass S over the interior dofs, summing only the
    elements in `elem_subset` (all elements when None).  With a subset this
    is the element-restricted ("Neumann") form a_D, (.,.)_D of Eq. 2.18."""
    dofs = dof_map(is_boundary)
    n = int((is_boundary == 0).sum())
    if elem_subset is not None:
        elems = elems[elem_subset]
        coeff = coeff[elem_subset]
    K, M = element_matrices(xyz, elems, coeff)
    nv = elems.shape[1]
    rows = np.repeat(dofs[elems], nv, axis=1).ravel()
    cols = np.tile(dofs[elems], (1, nv)).ravel()
    keep = (rows >= 0) & (cols >= 0)
    A = sp.csr_matrix((K.ravel()[keep], (rows[keep], cols[keep])), shape=(n, n))
    S = sp.csr_matrix((M.ravel()[keep], (rows[keep], cols[keep])), shape=(n, n))
    A.sum_duplicates()
    S.sum_duplicates()
    return A, S


def helmholtz_matrices(xyz, elems, coeff, is_boundary, k):
    """B = A - k^2 S (Eq. 2.12) and D_k = A + k^2 S (Prop. 2.6)."""
    A, S = assemble(xyz, elems, coeff, is_boundary)
    return (A - k * k * S).tocsr(), (A + k * k * S).tocsr(), A, S


def full_mass(xyz, elems):
    """Mass matrix over all nodes (Dirichlet nodes included)."""
    _, M = element_matrices(xyz, elems, np.ones(elems.shape[0]))
    nv = elems.shape[1]
    rows = np.repeat(elems, nv, axis=1).ravel()
    cols = np.tile(elems, (1, nv)).ravel()
    Mf = sp.csr_matrix((M.ravel(), (rows, cols)), shape=(xyz.shape[0],) * 2)
    Mf.sum_duplicates()
    return Mf


def load_vector_nodal(xyz, elems, is_boundary, f_nodal):
    """(f, phi_i) for the P1 interpolant of f (Eq. 2.12's right-hand side);
    exact when f itself is piecewise linear, e.g. f = 1."""
    dofs = dof_map(is_boundary)
    full = full_mass(xyz, elems) @ f_nodal
    return full[dofs >= 0]


# Dunavant's 7-point triangle rule, exact for polynomials of degree 5
# (barycentric points, weights summing to 1).
_A1, _B1 = 0.059715871789770, 0.470142064105115
_A2, _B2 = 0.797426985353087, 0.101286507323456
_DUN7_PTS = np.array([[1 / 3, 1 / 3, 1 / 3],
                      [_A1, _B1, _B1], [_B1, _A1, _B1], [_B1, _B1, _A1],
                      [_A2, _B2, _B2], [_B2, _A2, _B2], [_B2, _B2, _A2]])
_DUN7_W = np.array([0.225] + [0.132394152788506] * 3 + [0.125939180544827] * 3)


def load_vector_quadrature(xyz, elems, is_boundary, f):
    """(f, phi_i) for a smooth 2D source f(x, y) by the degree-5 rule."""
    assert xyz.shape[1] == 2
    vol, _ = barycentric_gradients(xyz, elems)
    P = xyz[elems]                                          # (ne, 3, 2)
    pts = np.einsum("qi,eid->eqd", _DUN7_PTS, P)            # (ne, 7, 2)
    fv = f(pts[..., 0], pts[..., 1])                        # (ne, 7)
    contrib = np.einsum("q,eq,qi->ei", _DUN7_W, fv, _DUN7_PTS) * vol[:, None]
    full = np.zeros(xyz.shape[0])
    np.add.at(full, elems.ravel(), contrib.ravel())
    return full[dof_map(is_boundary) >= 0]
