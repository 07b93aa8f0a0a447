"""Overlapping subdomains, dof sets and the partition of unity (oracle).

* Def. 2.3: a subdomain D' made of elements is extended by one layer to the
  interior of the union of the supports of every basis function phi_l of V^h
  whose support meets D'.  For P1, supp(phi_l) meets the open set D' exactly
  when node l is a vertex of an element of D', and supp(phi_l) is the star of
  l (the elements having l as a vertex).  Only interior nodes index basis
  functions of V^h, so only they extend the set.  Layers are applied
  recursively.  The elements of D' are kept (an element none of whose
  vertices is interior carries no basis function and does not change any
  matrix).
* Def. 3.2: ovdof(D) = dofs whose support meets D (interior vertices of D's
  elements); dof(D) = dofs whose support lies in the closure of D (interior
  nodes whose whole star is inside D).
* Def. 2.7: mu_l = number of subdomains having l in dof(D_i); the local
  partition of unity Xi_D weights dof l by 1/mu_l on dof(D) and by 0 on
  ovdof(D) \\ dof(D).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp

from .fem import dof_map


def node_element_incidence(elems: np.ndarray, n_nodes: int) -> sp.csr_matrix:
    """Sparse (n_nodes x n_elems) 0/1 matrix: node is a vertex of element."""
    ne, nv = elems.shape
    rows = elems.ravel()
    cols = np.repeat(np.arange(ne), nv)
    return sp.csr_matrix((np.ones(rows.size, dtype=np.int8), (rows, cols)), shape=(n_nodes, ne))


@dataclass
class Subdomain:
    elems: np.ndarray     # element ids of the overlapping subdomain (sorted)
    dof: np.ndarray       # global dof ids of dof(Omega_i), increasing   (I_i)
    ovdof: np.ndarray     # global dof ids of ovdof(Omega_i), increasing (O_i)


def extend_by_layers(elems, is_boundary, elem_set: np.ndarray, layers: int, inc=None, within=None) -> np.ndarray:
    """Def. 2.3 applied `layers` times to a boolean element mask; with `within` (a boolean element mask),
    in the mesh of that region: each layer keeps only the elements of `within`."""
    n_nodes = is_boundary.size
    if inc is None:
        inc = node_element_incidence(elems, n_nodes)
    interior = is_boundary == 0
    cur = elem_set.astype(bool).copy()
    for _ in range(layers):
        touched = (inc @ cur.astype(np.int8)) > 0            # nodes that are vertices of cur
        grow_nodes = touched & interior                       # basis functions of V^h meeting cur
        star_hit = (inc.T @ grow_nodes.astype(np.int8)) > 0   # elements in those supports
        cur = cur | star_hit
        if within is not None:
            cur &= within
    return cur


def subdomain_of(mask, inc, dofs, interior, star_size) -> "Subdomain":
    """dof and ovdof (Def. 3.2) of the overlapping subdomain with element mask `mask`."""
    in_star = np.asarray(inc @ mask.astype(np.int64)).ravel()     # elements of the star inside D
    ov_nodes = np.flatnonzero(interior & (in_star > 0))
    dof_nodes = np.flatnonzero(interior & (in_star == star_size))
    return Subdomain(np.flatnonzero(mask), np.sort(dofs[dof_nodes]), np.sort(dofs[ov_nodes]))


def decompose(xyz, elems, is_boundary, elem_to_sub, n_sub: int, overlap: int):
    """Overlapping subdomains (Def. 2.3) with their dof/ovdof (Def. 3.2) and mu (Def. 2.7)."""
    n_nodes = is_boundary.size
    inc = node_element_incidence(elems, n_nodes)
    dofs = dof_map(is_boundary)
    interior = is_boundary == 0
    star_size = np.asarray(inc.sum(axis=1)).ravel()
    subs = []
    mu = np.zeros(int(interior.sum()), dtype=np.int64)
    for i in range(n_sub):
        mask = extend_by_layers(elems, is_boundary, elem_to_sub == i, overlap, inc)
        sd = subdomain_of(mask, inc, dofs, interior, star_size)
        mu[sd.dof] += 1
        subs.append(sd)
    return subs, mu


def decompose_nested(xyz, elems, is_boundary, elem_to_sub, n_sub: int, overlap: int, elem_to_fine,
                     fine_overlap: int):
    """The two nested decompositions of Sec. 2.3.  Coarse: the subdomains Omega_i^c of `decompose`.
    Fine: inside each Omega_i^c, its elements grouped by their label in `elem_to_fine` (a partition of
    Omega_i^c into Q_i pieces), each piece extended `fine_overlap` times by Def. 2.3 in the mesh of
    Omega_i^c, so that Omega_i^c is the union of its fine subdomains Omega^f_{i,j}.  A fine subdomain
    without a dof (a sliver of Omega_i^c) spans the zero space and is left out.
    Returns (coarse subdomains, mu^c, fine subdomains, parent coarse index of each, mu^f)."""
    coarse, mu_c = decompose(xyz, elems, is_boundary, elem_to_sub, n_sub, overlap)
    n_nodes = is_boundary.size
    inc = node_element_incidence(elems, n_nodes)
    dofs = dof_map(is_boundary)
    interior = is_boundary == 0
    star_size = np.asarray(inc.sum(axis=1)).ravel()
    ne = elems.shape[0]
    fine, parent = [], []
    mu_f = np.zeros(int(interior.sum()), dtype=np.int64)
    for i, sd in enumerate(coarse):
        cmask = np.zeros(ne, dtype=bool)
        cmask[sd.elems] = True
        for g in np.unique(elem_to_fine[sd.elems]):
            piece = cmask & (elem_to_fine == g)
            mask = extend_by_layers(elems, is_boundary, piece, fine_overlap, inc, within=cmask)
            fd = subdomain_of(mask, inc, dofs, interior, star_size)
            if fd.dof.size == 0:
                continue
            mu_f[fd.dof] += 1
            fine.append(fd)
            parent.append(i)
    return coarse, mu_c, fine, np.array(parent, dtype=np.int64), mu_f


def multiplicity_lambda(elems, subs, n_elems) -> int:
    """Lambda of Sec. 2.4: the largest number of subdomains sharing an element."""
    cnt = np.zeros(n_elems, dtype=np.int64)
    for s in subs:
        cnt[s.elems] += 1
    return int(cnt.max())


def pou_weights(sd: Subdomain, mu: np.ndarray) -> np.ndarray:
    """Diagonal of Xi_i on ovdof(Omega_i): 1/mu_l on dof, 0 elsewhere (Def. 2.7)."""
    w = np.zeros(sd.ovdof.size)
    pos = np.searchsorted(sd.ovdof, sd.dof)
    w[pos] = 1.0 / mu[sd.dof]
    return w
