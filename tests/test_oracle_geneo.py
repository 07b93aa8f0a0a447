"""Pins of the oracle's H_k-GenEO eigenproblem (Eq. 5.12) and coarse space
(Def. 5.1) against independent routes: QZ on the unreduced pencil, inertia
counts (Sylvester / Haynsworth) from an independent LDL^T, the Moebius map of
the (K, M) pencil for one subdomain, and the residual of the unreduced
definition."""
import numpy as np
import pytest
import scipy.linalg as sla

from oracle import decomposition as D
from oracle import fem, geneo
from paper_2406_06283_gb300 import workloads as W


def _pencils(cells=8, parts=2, k=5.0, ov=1, checker=0):
    p = W.small_problem(cells=cells, parts=parts, k=k, overlap=ov, checker=checker)
    m = p.mesh
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, p.elem_to_sub, p.n_sub, ov)
    out = []
    for sd in subs:
        BN, C, w = geneo.local_pencil(m.xyz, m.elems, p.coeff, m.is_boundary, p.k, sd, mu)
        out.append((BN, C, w))
    return out


def _neg_count(Mat):
    # inertia from an independent symmetric indefinite factorisation
    lu, d, perm = sla.ldl(Mat, lower=True)
    return int(np.count_nonzero(np.linalg.eigvalsh(d) < 0))


@pytest.mark.parametrize("checker", [0, 2])
def test_finite_spectrum_matches_qz(checker):
    for BN, C, w in _pencils(checker=checker):
        ev = geneo.local_eigen(BN, C, w, tau=0.5)
        qz = geneo.finite_eigenvalues_qz(BN, C)
        assert qz.size == ev.lam.size
        np.testing.assert_allclose(ev.lam, qz, rtol=1e-8, atol=1e-9)


@pytest.mark.parametrize("sigma", [-0.5, 0.0, 0.3, 0.5, 0.9, 2.0])
def test_count_below_sigma_equals_inertia(sigma):
    # Haynsworth: In(B^N - sigma C) = In(B^N_GG) + In(S - sigma C_II), and by
    # Sylvester #neg(S - sigma C_II) = #{lambda < sigma} since C_II is SPD.
    for BN, C, w in _pencils(cells=12, parts=2, k=7.0, ov=2, checker=2):
        ev = geneo.local_eigen(BN, C, w, tau=0.5)
        G = w == 0
        want = _neg_count(BN - sigma * C) - _neg_count(BN[np.ix_(G, G)])
        assert int(np.count_nonzero(ev.lam < sigma)) == want


def test_unreduced_residual_and_normalisation():
    for BN, C, w in _pencils(cells=10, parts=2, k=6.0, ov=2, checker=2):
        ev = geneo.local_eigen(BN, C, w, tau=0.5)
        I, G = w > 0, w == 0
        for l in range(ev.lam.size):
            p = np.zeros(w.size)
            p[I] = ev.P[:, l]
            if G.any():
                p[G] = -np.linalg.solve(BN[np.ix_(G, G)], BN[np.ix_(G, I)] @ ev.P[:, l])
            r = BN @ p - ev.lam[l] * (C @ p)
            assert np.linalg.norm(r) <= 1e-9 * np.linalg.norm(BN @ p)
        # c(p_l, p_m) = delta_lm (the normalisation of the lemma on indefinite pencils)
        CII = C[np.ix_(I, I)]
        np.testing.assert_allclose(ev.P.T @ CII @ ev.P, np.eye(ev.lam.size), atol=1e-10)


@pytest.mark.parametrize("k", [3.0, 9.0])
def test_single_subdomain_moebius_map(k):
    # One subdomain = Omega: mu = 1 and ovdof = dof, so the pencil is
    # (K - k^2 M) p = lambda (K + k^2 M) p, i.e. lambda = (theta - k^2)/(theta + k^2)
    # for the eigenvalues theta of K p = theta M p.
    m = W.square_mesh(12)
    coeff = W.checkerboard(m, 3, W.stream_seed(11))
    e2s = np.zeros(m.n_elems, dtype=np.int32)
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, e2s, 1, 1)
    assert np.all(mu == 1) and subs[0].dof.size == subs[0].ovdof.size == m.n_dofs
    BN, C, w = geneo.local_pencil(m.xyz, m.elems, coeff, m.is_boundary, k, subs[0], mu)
    ev = geneo.local_eigen(BN, C, w, tau=0.5)
    A, S = fem.assemble(m.xyz, m.elems, coeff, m.is_boundary)
    theta = sla.eigh(A.toarray(), S.toarray(), eigvals_only=True)
    np.testing.assert_allclose(ev.lam, np.sort((theta - k * k) / (theta + k * k)), rtol=1e-9, atol=1e-12)


def test_selection_rule_ties():
    lam = np.array([-0.3, 0.1, 0.4999999999, 0.5000000001, 0.7])
    assert geneo.select_count(lam, 0.5) == 4
    assert geneo.select_count(np.array([-1.0, 0.2, 0.6]), 0.5) == 2
    assert geneo.select_count(np.array([0.6, 0.7]), 0.5) == 0


def test_coarse_vectors_are_pou_weighted():
    p = W.small_problem(cells=12, parts=2, k=6.0, overlap=2)
    m = p.mesh
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, p.elem_to_sub, p.n_sub, 2)
    BN, C, w = geneo.local_pencil(m.xyz, m.elems, p.coeff, m.is_boundary, p.k, subs[0], mu)
    ev = geneo.local_eigen(BN, C, w, tau=0.5)
    np.testing.assert_allclose(ev.Z, ev.P[:, : ev.m] / mu[subs[0].dof][:, None])
    assert np.all(ev.lam[: ev.m] < 0.5) and (ev.m == ev.lam.size or ev.lam[ev.m] >= 0.5)


def _dense_z_by_definition(subs, eigs, mu, n):
    """Def. 5.1 written out entry by entry: column l of subdomain i is E_i Xi_i p_l, i.e. zero
    off dof(Omega_i) and p_l[a] / mu_l at the a-th dof l of Omega_i (dofs in increasing order)."""
    cols = []
    for sd, ev in zip(subs, eigs):
        for l in range(ev.m):
            z = np.zeros(n)
            for a in range(sd.dof.size):
                g = int(sd.dof[a])
                z[g] = ev.P[a, l] / float(mu[g])
            cols.append(z)
    return np.stack(cols, axis=1) if cols else np.zeros((n, 0))


@pytest.mark.parametrize("cells,parts,ov,k", [(10, 2, 1, 5.0), (12, 3, 2, 7.0)])
def test_coarse_basis_matches_definition(cells, parts, ov, k):
    p = W.small_problem(cells=cells, parts=parts, k=k, overlap=ov, checker=2)
    m = p.mesh
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, p.elem_to_sub, p.n_sub, ov)
    eigs = []
    for sd in subs:
        BN, C, w = geneo.local_pencil(m.xyz, m.elems, p.coeff, m.is_boundary, p.k, sd, mu)
        eigs.append(geneo.local_eigen(BN, C, w, tau=0.5))
    assert sum(e.m for e in eigs) > 0
    want = _dense_z_by_definition(subs, eigs, mu, m.n_dofs)
    got = geneo.coarse_basis(subs, eigs, m.n_dofs).toarray()
    assert got.shape == want.shape
    # p / mu and p * (1 / mu) may differ in the last bit; a misplaced row or column differs by O(1)
    np.testing.assert_allclose(got, want, rtol=1e-15, atol=0.0)
    # each column is supported on its own subdomain's dof set only
    c0 = 0
    for sd, ev in zip(subs, eigs):
        off = np.setdiff1d(np.arange(m.n_dofs), sd.dof)
        assert np.all(got[off, c0:c0 + ev.m] == 0.0)
        c0 += ev.m
