"""GPU parity of the nested coarse/fine decompositions (Sec. 2.3) against the oracle
(oracle/decomposition.decompose_nested): the eigenproblems and the coarse space on the coarse subdomains, the
local solves on the fine ones.

Tolerances (as for the single decomposition, test_gpu_parity.py):
  fine decomposition   number of fine subdomains, sum of |dof(Omega^f)| and Lambda exact
  kept eigenvalues     m_i exact, lambda within 1e-9 (coarse subdomains)
  apply                FP64 1e-10, FP32 1e-4, split-BF16 (tensor-core sweeps) TOL_SPLIT
  FGMRES               FP64 counts inside the oracle's rounding range, FP32 within +-1; solution 1e-7;
                       true residual <= tol
  left D_k GMRES       FP64 counts inside the oracle's rounding range; solution 1e-7
"""
import numpy as np
import pytest

from oracle import solver as OS
from paper_2406_06283_gb300 import hk
from paper_2406_06283_gb300 import workloads as W
from test_gpu_parity import check_counts, oracle_count_range

pytestmark = pytest.mark.gpu


def _case(cells, parts, fine_parts, k, overlap, fine_overlap, checker, seed, dim=2):
    if dim == 2:
        p = W.small_problem(cells=cells, parts=parts, k=k, overlap=overlap, checker=checker, seed=seed)
    else:
        p = W.small_problem_3d(cells=cells, parts=parts, k=k, overlap=overlap, seed=seed)
    e2f = W.box_partition(p.mesh, fine_parts)
    return p, e2f, fine_parts ** dim, fine_overlap


CASES = {
    "h24_c3_f6_k12": _case(24, 3, 6, 12.0, 2, 1, 3, 8),
    "h40_c2_f8_k18": _case(40, 2, 8, 18.0, 2, 1, 4, 6),
    "h48_c4_f12_k20_fov2": _case(48, 4, 12, 20.0, 2, 2, 4, 9),
    "3d_h12_c2_f4_k6": _case(12, 2, 4, 6.0, 2, 1, 0, 10, dim=3),
}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p, e2f, nlab, fov = CASES[request.param]
    o = OS.setup_problem(p, nested=(e2f, fov))
    yield request.param, p, e2f, nlab, fov, o


def test_fine_decomposition_and_coarse_eigenproblems(case):
    name, p, e2f, nlab, fov, o = case
    h = hk.setup_problem_nested(p, e2f, nlab, fov)
    info = hk.hk_info(h)
    assert info["fine_subdomains"] == len(o.subs)
    assert info["fine_dof_total"] == sum(sd.dof.size for sd in o.subs)
    assert info["fine_lambda_elems"] == o.Lambda
    assert info["n_sub"] == len(o.coarse_subs) and info["n0"] == o.n0
    for i, ev in enumerate(o.eigs):
        lam, _, _ = hk.hk_get_eigen(h, i)
        assert lam.size == ev.m
        want = ev.lam[: ev.m]
        assert np.all(np.abs(lam - want) <= 1e-9 * np.maximum(np.abs(want), 1e-3))
    th = hk.hk_theory(h, 1.0, 0.0)
    assert th["Lambda"] == o.Lambda
    hk.hk_destroy(h)


@pytest.mark.parametrize("form", ["fp64", "fp32", "split"])
def test_nested_apply(case, form):
    from test_gpu_split_bf16 import TOL_SPLIT
    name, p, e2f, nlab, fov, o = case
    prec = {"fp64": hk.HK_FP64, "fp32": hk.HK_FP32_PRECOND, "split": hk.HK_SPLIT_BF16_PRECOND}[form]
    h = hk.setup_problem_nested(p, e2f, nlab, fov, precision=prec)
    if form == "split":
        hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    v = np.random.default_rng(3).standard_normal((5, o.n))
    z = hk.hk_apply_precond(h, v)
    hk.hk_destroy(h)
    want = np.stack([o.precond.apply(vi) for vi in v])
    tol = {"fp64": 1e-10, "fp32": 1e-4, "split": TOL_SPLIT}[form]
    err = np.linalg.norm(z - want, axis=1) / np.linalg.norm(want, axis=1)
    assert np.all(err <= tol), err


@pytest.mark.parametrize("form", ["fp64", "fp32"])
def test_nested_solve_parity(case, form):
    name, p, e2f, nlab, fov, o = case
    prec = hk.HK_FP64 if form == "fp64" else hk.HK_FP32_PRECOND
    h = hk.setup_problem_nested(p, e2f, nlab, fov, precision=prec)
    f = OS.load_vector(p)
    got = hk.hk_solve(h, f, p.tol)
    hk.hk_destroy(h)
    for r in range(f.shape[0]):
        rng_out = oracle_count_range(o, f[r], p.tol, key=("nested_" + name, r))
        check_counts("nested_" + name, r, form, got.iters[r], rng_out, widen=0 if form == "fp64" else 1)
        assert got.true_rel_res[r] <= p.tol
        assert _rel(got.u[r], rng_out[0].x) <= 1e-7


def test_nested_left_dk_gmres(case):
    from test_gpu_dk_gmres import dk_count_range
    name, p, e2f, nlab, fov, o = case
    h = hk.setup_problem_nested(p, e2f, nlab, fov)
    f = OS.load_vector(p)
    got, pc = hk.hk_solve_left_dk(h, f, p.tol)
    hk.hk_destroy(h)
    clean, lo, hi, _ = dk_count_range(o, f[0], p.tol, ("nested_" + name, 0))
    assert lo <= got.iters[0] <= hi, (int(got.iters[0]), lo, hi)
    assert pc[0] <= p.tol and _rel(got.u[0], clean.x) <= 1e-7


def test_nested_rejects_bad_arguments():
    p, e2f, nlab, fov = CASES["h24_c3_f6_k12"]
    with pytest.raises(hk.HKError):
        hk.setup_problem_nested(p, e2f, nlab - 1, fov)  # a label outside 0 .. n_fine_labels-1
    with pytest.raises(hk.HKError):
        hk.setup_problem_nested(p, e2f, nlab, 0)  # dofs on the piece interfaces lie in no fine dof set
