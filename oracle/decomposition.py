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


def extend_by_layers(elems, is_boundary, elem_set: np.ndarray, layers: int, inc=None) -> np.ndarray:
    """Def. 2.3 applied `layers` times to a boolean element mask."""
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
    return cur


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
        in_star = np.asarray(inc @ mask.astype(np.int64)).ravel()     # elements of the star inside D
        ov_nodes = np.flatnonzero(interior & (in_star > 0))
        dof_nodes = np.flatnonzero(interior & (in_star == star_size))
        sd = Subdomain(np.flatnonzero(mask), np.sort(dofs[dof_nodes]), np.sort(dofs[ov_nodes]))
        mu[sd.dof] += 1
        subs.append(sd)
    return subs, mu


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
