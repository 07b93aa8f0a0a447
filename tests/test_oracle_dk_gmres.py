"""Pins of the oracle's left-preconditioned GMRES in the D_k inner product (oracle/gmres_dk.py, the
setting of Thm. 3.1) and of its theory quantities.

* Equivalence with Euclidean GMRES: with D_k = L L^T (Cholesky), GMRES in the D_k inner product on
  A = M^{-1} B is Euclidean GMRES on L^T A L^{-T} with right-hand side L^T M^{-1} f, and the D_k norms
  of its residuals are the Euclidean norms of the transformed ones.  The transformed system is solved
  by scipy's GMRES (an independent implementation); the residual histories agree.
* Minimal residual property, by brute force: after m steps the residual is the least D_k-norm residual
  over the Krylov space span(r_0, A r_0, ..., A^{m-1} r_0), computed by a dense weighted least-squares
  solve on the explicit Krylov basis.
* A wrong inner product (Euclidean instead of D_k) changes the history, so the pins see the weight.
* Theory: Corollary 3.2's sufficient condition (H^f k <= C, (1 + C_stab)^2 k^2 <= C tau with
  2 Lambda^2 (2 + 3 Lambda^4 C)(2 sqrt(C) + 3 C) < 1) implies s < 1 and gamma > 0 with s below the
  corollary's bound; tau is the smallest left-out eigenvalue (lambda_{m_i} < tau_threshold <= tau).
"""
import numpy as np
import pytest
import scipy.linalg as sla
import scipy.sparse.linalg as spla

from oracle import gmres_dk as G
from oracle import solver as OS
from paper_2406_06283_gb300 import workloads as W


@pytest.fixture(scope="module")
def small():
    p = W.small_problem(cells=12, parts=2, k=8.0, overlap=1, checker=2)
    o = OS.setup_problem(p)
    f = OS.load_vector(p)[0]
    return p, o, f


def _dense_precond(o):
    n = o.n
    return np.stack([o.precond.apply(e) for e in np.eye(n)], axis=1)


def test_equals_euclidean_gmres_on_the_transformed_system(small):
    p, o, f = small
    Minv = _dense_precond(o)
    A = Minv @ o.B.toarray()
    D = o.Dk.toarray()
    L = np.linalg.cholesky(D)
    At = L.T @ A @ np.linalg.inv(L.T)
    bt = L.T @ (Minv @ f)
    got = G.gmres_left_dk(lambda v: o.B @ v, o.precond.apply, o.Dk, f, tol=1e-10, restart=200, max_iters=200)
    hist = []
    spla.gmres(At, bt, rtol=1e-10, atol=0.0, restart=200, maxiter=1, callback=lambda r: hist.append(r),
               callback_type="pr_norm")
    k = min(len(hist), len(got.history))
    assert k >= 10
    np.testing.assert_allclose(got.history[:k], hist[:k], rtol=1e-6)
    assert got.converged and abs(got.iters - len(hist)) <= 1
    # the solution of the preconditioned system is the solution of B u = f
    np.testing.assert_allclose(got.x, np.linalg.solve(o.B.toarray(), f), rtol=1e-7, atol=1e-9 * np.abs(got.x).max())


def test_minimal_residual_property_by_brute_force(small):
    p, o, f = small
    Minv = _dense_precond(o)
    A = Minv @ o.B.toarray()
    D = o.Dk.toarray()
    Lc = np.linalg.cholesky(D)
    r0 = Minv @ f
    beta0 = np.sqrt(r0 @ D @ r0)
    got = G.gmres_left_dk(lambda v: o.B @ v, o.precond.apply, o.Dk, f, tol=1e-14, restart=50, max_iters=8)
    K = [r0]
    for m in range(1, 8):
        Km = np.stack(K, axis=1)
        # min_y || r0 - A K y ||_D  =  min_y || L^T (r0 - A K y) ||_2
        y, *_ = sla.lstsq(Lc.T @ (A @ Km), Lc.T @ r0)
        res = r0 - A @ Km @ y
        want = np.sqrt(res @ D @ res) / beta0
        assert abs(got.history[m - 1] - want) <= 1e-8 * max(want, 1e-12), (m, got.history[m - 1], want)
        K.append(A @ K[-1] / np.linalg.norm(A @ K[-1]))


def test_the_weight_matters(small):
    p, o, f = small
    import scipy.sparse as sp
    dk = G.gmres_left_dk(lambda v: o.B @ v, o.precond.apply, o.Dk, f, tol=1e-10, restart=200, max_iters=200)
    eu = G.gmres_left_dk(lambda v: o.B @ v, o.precond.apply, sp.identity(o.n, format="csr"), f, tol=1e-10,
                         restart=200, max_iters=200)
    k = min(len(dk.history), len(eu.history))
    assert np.max(np.abs(np.array(dk.history[:k]) / np.array(eu.history[:k]) - 1.0)) > 1e-3


def test_restarted_solve_converges_to_the_same_solution(small):
    p, o, f = small
    a = G.gmres_left_dk(lambda v: o.B @ v, o.precond.apply, o.Dk, f, tol=1e-10, restart=5, max_iters=400)
    assert a.converged and a.pc_rel_res <= 1e-10
    np.testing.assert_allclose(a.x, np.linalg.solve(o.B.toarray(), f), rtol=1e-6, atol=1e-9 * np.abs(a.x).max())
    # restarts lose the Krylov space: never fewer iterations than the unrestarted solve
    b = G.gmres_left_dk(lambda v: o.B @ v, o.precond.apply, o.Dk, f, tol=1e-10, restart=200, max_iters=400)
    assert a.iters >= b.iters


def test_tau_is_the_smallest_left_out_eigenvalue(small):
    p, o, f = small
    tau = G.tau_next(o.eigs)
    assert tau >= p.tau
    assert any(abs(e.lam[e.m] - tau) == 0.0 for e in o.eigs if e.m < e.lam.size)
    for e in o.eigs:
        assert e.m == 0 or e.lam[e.m - 1] < p.tau


@pytest.mark.parametrize("Lam", [1, 2, 4])
def test_corollary_condition_implies_s_below_one(Lam):
    # the largest C of the form 10^-q meeting the corollary's smallness condition
    C = next(10.0 ** -q for q in np.arange(0, 20, 0.25)
             if 2 * Lam ** 2 * (2 + 3 * Lam ** 4 * 10.0 ** -q) * (2 * np.sqrt(10.0 ** -q) + 3 * 10.0 ** -q) < 1)
    bound = 2 * Lam ** 2 * (2 + 3 * Lam ** 4 * C) * (2 * np.sqrt(C) + 3 * C)
    rng = np.random.default_rng(Lam)
    for _ in range(200):
        k = 10 ** rng.uniform(0, 2)
        c_stab = 10 ** rng.uniform(-1, 1)
        H_f = C / k * rng.uniform(0.01, 1.0)            # H^f k <= C
        tau = (1 + c_stab) ** 2 * k * k / C * rng.uniform(1.0, 100.0)  # (1 + C_stab)^2 k^2 <= C tau
        t = G.theory(Lam, tau, k, H_f, c_stab)
        assert t["s"] <= bound * (1 + 1e-12) and t["s"] < 1 and t["gamma"] > 0 and t["guaranteed"]
    # and outside it the guarantee can fail
    t = G.theory(Lam, 1e-3, 10.0, 0.1, 1.0)
    assert t["s"] > 1 and t["gamma"] < 0 and not t["guaranteed"]
