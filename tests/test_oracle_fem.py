"""Pins of the oracle's P1 discretisation (Sec. 2.1, Eq. 2.11-2.12) against
closed forms that do not go through the oracle's own formulas."""
import numpy as np
import pytest
import scipy.sparse.linalg as spla

from oracle import fem
from paper_2406_06283_gb300 import workloads as W


@pytest.mark.parametrize("C", [16, 64])
def test_stiffness_sine_modes(C):
    # A = I on right triangles gives the 5-point stencil; sin(p pi x) sin(q pi y)
    # are eigenvectors with eigenvalue 4 sin^2(p pi h/2) + 4 sin^2(q pi h/2).
    m = W.square_mesh(C)
    A, S = fem.assemble(m.xyz, m.elems, np.ones(m.n_elems), m.is_boundary)
    inner = m.is_boundary == 0
    x, y = m.xyz[inner, 0], m.xyz[inner, 1]
    h = 1.0 / C
    for p in (1, 2, 3):
        for q in (1, 2, 3):
            v = np.sin(p * np.pi * x) * np.sin(q * np.pi * y)
            lam = 4 * np.sin(p * np.pi * h / 2) ** 2 + 4 * np.sin(q * np.pi * h / 2) ** 2
            np.testing.assert_allclose(A @ v, lam * v, atol=1e-12)


def test_mass_entries():
    C = 16
    h = 1.0 / C
    m = W.square_mesh(C)
    _, S = fem.assemble(m.xyz, m.elems, np.ones(m.n_elems), m.is_boundary)
    S = S.toarray()
    np.testing.assert_allclose(np.diag(S), h * h / 2, rtol=1e-13)
    # 7-point pattern: E, W, N, S, NE, SW each h^2/12
    nx = C - 1
    idx = lambda i, j: (j - 1) * nx + (i - 1)  # noqa: E731
    c = idx(5, 5)
    for (di, dj) in [(1, 0), (-1, 0), (0, 1), (0, -1), (1, 1), (-1, -1)]:
        assert S[c, idx(5 + di, 5 + dj)] == pytest.approx(h * h / 12, rel=1e-13)
    for (di, dj) in [(1, -1), (-1, 1), (2, 0)]:
        assert S[c, idx(5 + di, 5 + dj)] == 0.0
    assert np.count_nonzero(S[c]) == 7
    Mf = fem.full_mass(m.xyz, m.elems)
    inner = m.is_boundary == 0
    np.testing.assert_allclose(np.asarray(Mf.sum(axis=1)).ravel()[inner], h * h, rtol=1e-12)


@pytest.mark.parametrize("mesh", [W.square_mesh(8), W.cube_mesh(4)])
def test_mass_integrates_linear_products(mesh):
    # v^T M w = int v w exactly for P1 v, w; on the unit box int x y = 1/4, int x^2 = 1/3.
    Mf = fem.full_mass(mesh.xyz, mesh.elems)
    x, y = mesh.xyz[:, 0], mesh.xyz[:, 1]
    one = np.ones(mesh.n_nodes)
    assert one @ (Mf @ one) == pytest.approx(1.0, rel=1e-13)
    assert x @ (Mf @ y) == pytest.approx(0.25, rel=1e-13)
    assert x @ (Mf @ x) == pytest.approx(1.0 / 3.0, rel=1e-13)


@pytest.mark.parametrize("mesh", [W.square_mesh(8), W.cube_mesh(4)])
def test_stiffness_of_linear_functions(mesh):
    # a(x, x) = int |grad x|^2 = 1 over the unit box; constants are in the kernel.
    from oracle.fem import element_matrices
    K, _ = element_matrices(mesh.xyz, mesh.elems, np.ones(mesh.n_elems))
    x = mesh.xyz[:, 0][mesh.elems]
    one = np.ones_like(x)
    assert np.einsum("ei,eij,ej->", x, K, x) == pytest.approx(1.0, rel=1e-12)
    np.testing.assert_allclose(np.einsum("eij,ej->ei", K, one), 0.0, atol=1e-12)


def test_load_vector_f_equals_one():
    C = 32
    m = W.square_mesh(C)
    f = fem.load_vector_nodal(m.xyz, m.elems, m.is_boundary, np.ones(m.n_nodes))
    np.testing.assert_allclose(f, 1.0 / C ** 2, rtol=1e-12)


@pytest.mark.parametrize("k", [1.0, 2.0])
def test_manufactured_solution_rate(k):
    # u = sin(pi x) sin(pi y) solves -Lap u - k^2 u = (2 pi^2 - k^2) u; the nodal
    # error of P1 on these meshes decays like h^2.
    errs, hs = [], []
    for C in (16, 32, 64, 128):
        m = W.square_mesh(C)
        B, _, _, _ = fem.helmholtz_matrices(m.xyz, m.elems, np.ones(m.n_elems), m.is_boundary, k)
        src = lambda x, y: (2 * np.pi ** 2 - k * k) * np.sin(np.pi * x) * np.sin(np.pi * y)  # noqa: E731
        f = fem.load_vector_quadrature(m.xyz, m.elems, m.is_boundary, src)
        u = spla.spsolve(B.tocsc(), f)
        inner = m.is_boundary == 0
        ue = np.sin(np.pi * m.xyz[inner, 0]) * np.sin(np.pi * m.xyz[inner, 1])
        errs.append(np.sqrt(np.sum((u - ue) ** 2)) / C)
        hs.append(1.0 / C)
    rates = np.diff(np.log(errs)) / np.diff(np.log(hs))
    assert np.all((rates > 1.8) & (rates < 2.2)), rates


def test_quadrature_rule_exactness():
    # Dunavant-7 integrates degree-5 monomials on the reference triangle exactly:
    # int x^a y^b = a! b! / (a+b+2)!.
    from math import factorial
    xyz = np.array([[0.0, 0.0], [1.0, 0.0], [0.0, 1.0]])
    elems = np.array([[0, 1, 2]])
    vol, _ = fem.barycentric_gradients(xyz, elems)
    pts = np.einsum("qi,id->qd", fem._DUN7_PTS, xyz)
    for a in range(6):
        for b in range(6 - a):
            val = vol[0] * np.sum(fem._DUN7_W * pts[:, 0] ** a * pts[:, 1] ** b)
            exact = factorial(a) * factorial(b) / factorial(a + b + 2)
            assert val == pytest.approx(exact, rel=1e-12, abs=1e-15)
