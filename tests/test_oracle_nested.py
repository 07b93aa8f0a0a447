"""Pins of the oracle's nested coarse/fine decompositions (Sec. 2.3) and their preconditioner.

* Structure: every fine subdomain lies in its coarse parent and the fine subdomains of Omega_i^c cover it
  (Omega_i^c = union_j Omega^f_{i,j}); without fine overlap the pieces of Omega_i^c are disjoint and
  partition its elements.
* Degenerate case: one fine label everywhere and no fine overlap gives Q_i = 1 and Omega^f_{i,1} =
  Omega_i^c, and the nested preconditioner is the single-decomposition one (bit for bit: the same
  operations on the same matrices).
* The nested preconditioner entry by entry from its definition, Eq. 2.22-2.23 with the fine restrictions:
  sum_{i,j} R_{ij}^T B_{ij}^{-1} R_{ij} + Z E^{-1} Z^T with Z from the coarse subdomains' eigenvectors.
* Lemma 3.4: if H^f k < sqrt(2) (A >= 1), every fine local matrix B^f_{i,j} is positive definite; and a
  case that breaks the condition has an indefinite one, so the check can fail.
* Lambda counts the fine subdomains sharing an element.
"""
import numpy as np

from oracle import decomposition as OD
from oracle import fem as OF
from oracle import solver as OS
from paper_2406_06283_gb300 import workloads as W


def _nested_case(cells=24, parts=3, fine_parts=6, k=12.0, overlap=2, fine_overlap=1, seed=8, checker=3):
    p = W.small_problem(cells=cells, parts=parts, k=k, overlap=overlap, checker=checker, seed=seed)
    e2f = W.box_partition(p.mesh, fine_parts)
    return p, e2f, fine_overlap


def test_fine_subdomains_cover_their_coarse_parent():
    p, e2f, fo = _nested_case()
    m = p.mesh
    for fov in (0, fo):
        coarse, mu_c, fine, parent, mu_f = OD.decompose_nested(m.xyz, m.elems, m.is_boundary, p.elem_to_sub,
                                                              p.n_sub, p.overlap, e2f, fov)
        for i, sd in enumerate(coarse):
            kids = [fine[j] for j in np.flatnonzero(parent == i)]
            assert len(kids) >= 2  # Q_i > 1: the fine labels split every coarse subdomain here
            union = np.unique(np.concatenate([f.elems for f in kids]))
            cset = set(sd.elems.tolist())
            assert all(set(f.elems.tolist()) <= cset for f in kids)
            # slivers without dofs are left out, so the union may miss only elements of dof-less pieces
            missing = np.setdiff1d(sd.elems, union)
            assert missing.size == 0 or fov == 0
            if fov == 0:
                allel = np.concatenate([f.elems for f in kids])
                assert np.unique(allel).size == allel.size  # disjoint pieces
        assert np.all(mu_c >= 1)
        # with fine overlap every dof lies in some fine dof set; without it the dofs on the interfaces
        # between pieces lie in none (their stars cross two pieces)
        assert np.all(mu_f >= 1) if fov > 0 else np.any(mu_f == 0)


def test_one_fine_label_is_the_single_decomposition():
    p = W.small_problem(cells=24, parts=3, k=12.0, overlap=2, checker=3, seed=8)
    e2f = np.zeros(p.mesh.n_elems, dtype=np.int64)
    a = OS.setup_problem(p)
    b = OS.setup_problem(p, nested=(e2f, 0))
    assert len(b.subs) == len(a.subs)
    for sa, sb in zip(a.subs, b.subs):
        np.testing.assert_array_equal(sa.elems, sb.elems)
        np.testing.assert_array_equal(sa.dof, sb.dof)
    v = np.random.default_rng(1).standard_normal(a.n)
    np.testing.assert_array_equal(a.precond.apply(v), b.precond.apply(v))


def test_nested_preconditioner_matches_its_definition():
    p, e2f, fo = _nested_case()
    o = OS.setup_problem(p, nested=(e2f, fo))
    n = o.n
    B = o.B.toarray()
    M = np.zeros((n, n))
    for fd in o.subs:
        R = np.zeros((fd.dof.size, n))
        R[np.arange(fd.dof.size), fd.dof] = 1.0
        M += R.T @ np.linalg.solve(R @ B @ R.T, R)
    # coarse vectors from the coarse subdomains: Xi_i p_l = p_l / mu^c on dof(Omega_i^c) (Def. 5.1)
    cols = []
    for sd, ev in zip(o.coarse_subs, o.eigs):
        for l in range(ev.m):
            z = np.zeros(n)
            z[sd.dof] = ev.P[:, l] / o.mu_c[sd.dof]
            cols.append(z)
    Z = np.stack(cols, axis=1)
    M += Z @ np.linalg.solve(Z.T @ B @ Z, Z.T)
    V = np.random.default_rng(2).standard_normal((3, n))
    for v in V:
        np.testing.assert_allclose(o.precond.apply(v), M @ v, rtol=1e-9, atol=1e-11 * np.abs(M @ v).max())
    assert o.Lambda == OD.multiplicity_lambda(p.mesh.elems, o.subs, p.mesh.n_elems)
    assert o.Lambda > OD.multiplicity_lambda(p.mesh.elems, o.coarse_subs, p.mesh.n_elems) - 1


def _fine_min_eigs(p, e2f, fo):
    m = p.mesh
    _, _, fine, _, _ = OD.decompose_nested(m.xyz, m.elems, m.is_boundary, p.elem_to_sub, p.n_sub, p.overlap,
                                           e2f, fo)
    B, _, _, _ = OF.helmholtz_matrices(m.xyz, m.elems, p.coeff, m.is_boundary, p.k)
    B = B.tocsr()
    out, diam = [], 0.0
    for fd in fine:
        out.append(np.linalg.eigvalsh(B[fd.dof][:, fd.dof].toarray())[0])
        x = m.xyz[np.unique(m.elems[fd.elems])]
        diam = max(diam, float(np.max(np.linalg.norm(x[:, None, :] - x[None, :, :], axis=2))))
    return np.array(out), diam


def test_lemma_3_4_small_fine_subdomains_are_positive_definite():
    # fine boxes of 4 cells + 1 layer on h = 1/24: diameter about 0.35; k = 3.5 gives H^f k < sqrt(2)
    p, e2f, fo = _nested_case(k=3.5, checker=3)
    lam, H = _fine_min_eigs(p, e2f, fo)
    assert H * p.k < np.sqrt(2.0)
    assert np.all(lam > 0)
    # coarse-sized local problems at a larger k break the condition, and an indefinite one appears
    q = W.small_problem(cells=24, parts=2, k=14.0, overlap=2, checker=3, seed=8)
    e1 = np.zeros(q.mesh.n_elems, dtype=np.int64)
    lam2, H2 = _fine_min_eigs(q, e1, 0)
    assert H2 * q.k > np.sqrt(2.0) and np.any(lam2 < 0)
