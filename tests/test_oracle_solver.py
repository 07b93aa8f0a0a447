"""Pins of the oracle's preconditioners (Eq. 2.22, 2.23) and FGMRES by special
cases whose iteration counts are fixed by linear algebra, and by dense solves."""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from oracle import decomposition as D
from oracle import fem, geneo, schwarz, solver
from oracle.fgmres import fgmres
from paper_2406_06283_gb300 import workloads as W


def test_gmres_distinct_eigenvalues():
    # GMRES on a diagonalisable matrix with d distinct eigenvalues ends in d steps.
    rng = np.random.default_rng(0)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    A = Q @ np.diag(np.repeat([1.0, -2.0, 5.0], [10, 20, 10])) @ Q.T
    r = fgmres(lambda v: A @ v, lambda v: v, rng.standard_normal(40), tol=1e-12, restart=50)
    assert r.converged and r.iters == 3


def test_gmres_restart_and_history():
    rng = np.random.default_rng(1)
    A = np.diag(np.linspace(1, 10, 200)) + 0.1 * rng.standard_normal((200, 200)) / 14
    f = rng.standard_normal(200)
    r = fgmres(lambda v: A @ v, lambda v: v, f, tol=1e-10, restart=7, max_iters=500)
    assert r.converged
    np.testing.assert_allclose(A @ r.x, f, atol=1e-9 * np.linalg.norm(f))
    assert len(r.history) == r.iters and r.history[-1] <= 1e-10
    assert np.all(np.diff(r.history[:7]) <= 1e-15)   # GMRES residuals never grow within a cycle


def _one_sub_problem(k=6.0):
    p = W.small_problem(cells=12, parts=1, k=k, overlap=1, checker=2)
    return p


def test_one_subdomain_one_level_is_exact():
    p = _one_sub_problem()
    h = solver.setup_problem(p, levels="one")
    r = solver.solve(h, p.rhs, tol=1e-10)[0]
    assert r.iters == 1 and r.converged


def test_one_subdomain_two_level_two_steps():
    # M^{-1} B = I + P with P a projection: minimal polynomial of degree 2.
    p = _one_sub_problem(k=15.0)
    h = solver.setup_problem(p, levels="two")
    assert h.n0 > 0
    r = solver.solve(h, p.rhs, tol=1e-10)[0]
    assert r.iters <= 2 and r.converged


def test_full_coarse_space_is_exact():
    # tau = +inf keeps every eigenvector; a column basis of Z spans R^n (partition
    # of unity), so the coarse term alone is B^{-1}: one iteration.
    p = W.small_problem(cells=10, parts=2, k=5.0, overlap=1, checker=2)
    m = p.mesh
    B, _, _, _ = fem.helmholtz_matrices(m.xyz, m.elems, p.coeff, m.is_boundary, p.k)
    subs, mu = D.decompose(m.xyz, m.elems, m.is_boundary, p.elem_to_sub, p.n_sub, 1)
    eigs = []
    for sd in subs:
        BN, C, w = geneo.local_pencil(m.xyz, m.elems, p.coeff, m.is_boundary, p.k, sd, mu)
        eigs.append(geneo.local_eigen(BN, C, w, tau=np.inf))
    Z = geneo.coarse_basis(subs, eigs, B.shape[0]).toarray()
    Q, R, piv = sla.qr(Z, mode="economic", pivoting=True)
    rank = int(np.count_nonzero(np.abs(np.diag(R)) > 1e-10 * abs(R[0, 0])))
    assert rank == B.shape[0]
    pc = schwarz.AdditiveSchwarz(B, subs, mu, sp.csr_matrix(Q[:, :rank]), levels="coarse")
    r = fgmres(lambda v: B @ v, pc.apply, p.rhs[0], tol=1e-10)
    assert r.iters == 1 and r.converged


def test_coarse_term_depends_only_on_span():
    p = W.small_problem(cells=12, parts=2, k=6.0, overlap=2, checker=2)
    h = solver.setup_problem(p)
    rng = np.random.default_rng(3)
    Zr = h.Z.toarray().copy()
    c0 = 0
    for mi in h.m_i:
        G, _ = np.linalg.qr(rng.standard_normal((mi, mi)))
        Zr[:, c0:c0 + mi] = Zr[:, c0:c0 + mi] @ G
        c0 += mi
    pc2 = schwarz.AdditiveSchwarz(h.B, h.subs, h.mu, sp.csr_matrix(Zr), levels="two")
    v = rng.standard_normal(h.n)
    np.testing.assert_allclose(pc2.apply(v), h.precond.apply(v), rtol=1e-9, atol=1e-12)


@pytest.mark.parametrize("levels", ["one", "two"])
@pytest.mark.parametrize("cells,parts,k", [(12, 2, 5.0), (16, 3, 9.0)])
def test_solution_matches_dense_solve(levels, cells, parts, k):
    p = W.small_problem(cells=cells, parts=parts, k=k, overlap=1, checker=2)
    h = solver.setup_problem(p, levels=levels)
    r = solver.solve(h, p.rhs, tol=1e-12)[0]
    u = np.linalg.solve(h.B.toarray(), p.rhs[0])
    assert np.linalg.norm(r.x - u) <= 1e-9 * np.linalg.norm(u)


def test_preconditioner_matches_dense_definition():
    # Eq. 2.22-2.23 written with dense Boolean restriction matrices.
    p = W.small_problem(cells=10, parts=2, k=4.0, overlap=1, checker=2)
    h = solver.setup_problem(p)
    Bd = h.B.toarray()
    n = h.n
    M = np.zeros((n, n))
    for sd in h.subs:
        R = np.zeros((sd.dof.size, n))
        R[np.arange(sd.dof.size), sd.dof] = 1.0
        M += R.T @ np.linalg.inv(R @ Bd @ R.T) @ R
    Z = h.Z.toarray()
    M += Z @ np.linalg.inv(Z.T @ Bd @ Z) @ Z.T
    v = np.random.default_rng(5).standard_normal(n)
    np.testing.assert_allclose(h.precond.apply(v), M @ v, rtol=1e-10, atol=1e-12)


def test_singular_local_detected():
    # Remark after Lemma 3.4: the local problem is singular when k^2 is a
    # Dirichlet eigenvalue of the subdomain.  One subdomain = Omega, k^2 = theta_1.
    p = W.small_problem(cells=8, parts=1, k=1.0, overlap=1)
    m = p.mesh
    A, S = fem.assemble(m.xyz, m.elems, p.coeff, m.is_boundary)
    theta = sla.eigh(A.toarray(), S.toarray(), eigvals_only=True)
    p.k = float(np.sqrt(theta[0]))
    with pytest.raises(schwarz.SingularLocal):
        solver.setup_problem(p, levels="one")


def test_load_vector_helper_f1():
    p = W.config_c1()
    f = solver.load_vector(p)
    np.testing.assert_allclose(f, 1.0 / 64 ** 2, rtol=1e-12)


@pytest.mark.parametrize("levels", ["one", "two", "coarse"])
@pytest.mark.parametrize("weighting", ["as", "ras_pou"])
def test_preconditioner_variants_match_dense_definition(levels, weighting):
    """Every variant of the preconditioner written with dense matrices built from the
    definitions: R_i the Boolean restriction to dof(Omega_i) (Sec. 2.3), the local term
    R_i^T W_i B_i^{-1} R_i with W_i = I (Eq. 2.22) or diag(1/mu) (the partition-of-unity
    variant), and the coarse term Z (Z^T B Z)^{-1} Z^T (Eq. 2.23) with Z assembled entry by
    entry from Def. 5.1 (column l of subdomain i is p_l / mu on dof(Omega_i), zero elsewhere)."""
    p = W.small_problem(cells=12, parts=3, k=6.0, overlap=2, checker=2, seed=4)
    h = solver.setup_problem(p, levels=levels, weighting=weighting)
    Bd = h.B.toarray()
    n = h.n
    M = np.zeros((n, n))
    if levels in ("one", "two"):
        for sd in h.subs:
            R = np.zeros((sd.dof.size, n))
            for a in range(sd.dof.size):
                R[a, sd.dof[a]] = 1.0
            Wt = np.diag(1.0 / h.mu[sd.dof]) if weighting == "ras_pou" else np.eye(sd.dof.size)
            M += R.T @ Wt @ np.linalg.inv(R @ Bd @ R.T) @ R
    if levels in ("two", "coarse"):
        subs, mu = D.decompose(p.mesh.xyz, p.mesh.elems, p.mesh.is_boundary, p.elem_to_sub, p.n_sub, p.overlap)
        cols = []
        for sd in subs:
            BN, C, w = geneo.local_pencil(p.mesh.xyz, p.mesh.elems, p.coeff, p.mesh.is_boundary, p.k, sd, mu)
            ev = geneo.local_eigen(BN, C, w, p.tau)
            for l in range(ev.m):
                z = np.zeros(n)
                for a in range(sd.dof.size):
                    z[sd.dof[a]] = ev.P[a, l] / mu[sd.dof[a]]
                cols.append(z)
        Z = np.stack(cols, axis=1)
        assert Z.shape[1] == h.n0 > 0
        M += Z @ np.linalg.inv(Z.T @ Bd @ Z) @ Z.T
    v = np.random.default_rng(6).standard_normal(n)
    np.testing.assert_allclose(h.precond.apply(v), M @ v, rtol=1e-9, atol=1e-11 * np.abs(M @ v).max())
