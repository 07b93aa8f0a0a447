"""GPU parity of the split-BF16 preconditioner form: the local block sweeps of Eq. 2.22 as
tensor-core products (tcgen05, BF16 pairs accumulated in FP32), the coarse correction of Eq. 2.23
in FP32, the Krylov method in FP64.

Tolerances (stated per result):
  apply, tensor-core sweeps     TOL_SPLIT relative to the oracle's FP64 apply (derivation below)
  apply, CUDA-core sweeps       bitwise equal to the FP32 form's apply (the same kernels on the same
                                FP32 records)
  FGMRES                        iterations within +-1 of the oracle's rounding range (the FP32
                                form's bar); solution 1e-7 relative; true residual <= tol

TOL_SPLIT.  Every record entry and every vector entry is held as a BF16 pair, whose relative
representation error is at most u = 2^-17 (two roundings to 8-bit significands), and a level product
drops the lo*lo term, also below u relative per term; the products accumulate in FP32.  The apply's
error is therefore a multiple of u set by the error growth through the dependent sweeps and by the
condition of the local matrices (measured on these problems: under 1 u, as the FP32 sweeps stay under
5 units of 2^-24).  TOL_SPLIT = 1e-3 (131 u) leaves room for longer sweep chains and worse-conditioned
local matrices than these.
"""
import numpy as np
import pytest

from oracle import solver as OS
from paper_2406_06283_gb300 import hk
from paper_2406_06283_gb300 import workloads as W
from test_gpu_parity import check_counts, oracle_count_range

pytestmark = pytest.mark.gpu

TOL_SPLIT = 1e-3

CASES = {
    "h16_p2_k6_ov1": W.small_problem(cells=16, parts=2, k=6.0, overlap=1, checker=2),
    "h24_p3_k12_ov2": W.small_problem(cells=24, parts=3, k=12.0, overlap=2, checker=3, seed=8),
    "h20_p3_k9_ov1_uneven": W.small_problem(cells=20, parts=3, k=9.0, overlap=1, checker=2, seed=5),
    "h40_p4_k18_ov2": W.small_problem(cells=40, parts=4, k=18.0, overlap=2, checker=4, seed=6, n_rhs=2),
    "h96_p3_k30_ov2": W.small_problem(cells=96, parts=3, k=30.0, overlap=2, checker=3, seed=14),
    "3d_h8_p2_k4_ov1": W.small_problem_3d(cells=8, parts=2, k=4.0, overlap=1),
    "3d_h12_p3_k6_ov2": W.small_problem_3d(cells=12, parts=3, k=6.0, overlap=2, seed=10),
}


def _rel(a, b):
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300)


def _rel_rows(a, b):
    return np.linalg.norm(a - b, axis=1) / np.maximum(np.linalg.norm(b, axis=1), 1e-300)


@pytest.fixture(scope="module", params=list(CASES))
def case(request):
    p = CASES[request.param]
    o = OS.setup_problem(p)
    h = hk.setup_problem(p, precision=hk.HK_SPLIT_BF16_PRECOND)
    yield request.param, p, o, h
    hk.hk_destroy(h)


def test_tensor_core_records_are_built(case):
    _, _, _, h = case
    info = hk.hk_info(h)
    assert info["precision"] == hk.HK_SPLIT_BF16_PRECOND
    assert info["tc_record_bytes"] > 0


@pytest.mark.parametrize("n_rhs", [1, 5, 16, 21])
def test_split_apply_matches_oracle(case, n_rhs):
    """1 and 5 right-hand sides fill part of the MMA's N = 16; 21 takes two CTA groups, the second
    with a ragged tail of 5."""
    _, _, o, h = case
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    v = np.random.default_rng(100 + n_rhs).standard_normal((n_rhs, o.n))
    z = hk.hk_apply_precond(h, v)
    assert hk.hk_info(h)["last_sweeps"] == hk.HK_SWEEPS_TENSOR_CORE
    want = np.stack([o.precond.apply(vi) for vi in v])
    err = _rel_rows(z, want)
    assert np.all(err <= TOL_SPLIT), err
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_AUTO)


def test_split_cuda_core_path_is_the_fp32_form(case):
    _, p, o, h = case
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_CUDA_CORE)
    v = np.random.default_rng(7).standard_normal((3, o.n))
    z = hk.hk_apply_precond(h, v)
    assert hk.hk_info(h)["last_sweeps"] == hk.HK_SWEEPS_CUDA_CORE
    h32 = hk.setup_problem(p, precision=hk.HK_FP32_PRECOND)
    z32 = hk.hk_apply_precond(h32, v)
    hk.hk_destroy(h32)
    np.testing.assert_array_equal(z, z32)
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_AUTO)


def test_split_solve_parity(case):
    name, p, o, h = case
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    f = OS.load_vector(p)
    got = hk.hk_solve(h, f, p.tol)
    for r in range(f.shape[0]):
        rng_out = oracle_count_range(o, f[r], p.tol, key=(name, r))
        check_counts(name, r, "split_bf16", got.iters[r], rng_out, widen=1)
        assert got.true_rel_res[r] <= p.tol
        assert _rel(got.u[r], rng_out[0].x) <= 1e-7
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_AUTO)


@pytest.mark.parametrize("shape", [(12, 12, 1), (12, 6, 1), (16, 8, 2)])
def test_split_apply_small_subdomains(shape):
    """Subdomains of 1 to 23 dofs: one level (the middle step alone), middle and bottom, short halves;
    records narrower than one 16-column MMA step and levels of one dof."""
    cells, parts, ov = shape
    p = W.small_problem(cells=cells, parts=parts, k=3.0, overlap=ov, checker=2)
    o = OS.setup_problem(p)
    v = np.random.default_rng(4).standard_normal((17, o.n))
    want = np.stack([o.precond.apply(vi) for vi in v])
    h = hk.setup_problem(p, precision=hk.HK_SPLIT_BF16_PRECOND)
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    z = hk.hk_apply_precond(h, v)
    hk.hk_destroy(h)
    assert np.all(_rel_rows(z, want) <= TOL_SPLIT)


def test_split_one_level_and_coarse_only():
    p = CASES["h24_p3_k12_ov2"]
    o1 = OS.setup_problem(p, levels="one")
    v = np.random.default_rng(9).standard_normal((4, o1.n))
    h = hk.setup_problem(p, precision=hk.HK_SPLIT_BF16_PRECOND, levels=hk.HK_ONE_LEVEL)
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    z = hk.hk_apply_precond(h, v)
    hk.hk_destroy(h)
    assert np.all(_rel_rows(z, np.stack([o1.precond.apply(vi) for vi in v])) <= TOL_SPLIT)
    # coarse only: no local sweeps, so no tensor-core records and the FP32 coarse correction
    h = hk.setup_problem(p, precision=hk.HK_SPLIT_BF16_PRECOND, levels=hk.HK_COARSE_ONLY)
    assert hk.hk_info(h)["tc_record_bytes"] == 0
    with pytest.raises(hk.HKError):
        hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    hk.hk_destroy(h)


def test_sweep_path_errors():
    p = CASES["h16_p2_k6_ov1"]
    h = hk.setup_problem(p, precision=hk.HK_FP32_PRECOND)
    with pytest.raises(hk.HKError) as e:
        hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    assert e.value.status == hk.HK_UNSUPPORTED
    with pytest.raises(hk.HKError) as e:
        hk.hk_set_sweep_path(h, 7)
    assert e.value.status == hk.HK_BAD_ARG
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_CUDA_CORE)
    hk.hk_destroy(h)


def test_split_apply_wide_3d_levels():
    """3D boxes of the serving operator's size (h = 1/32, 4x4x4 boxes, overlap 2): level sets wider than
    64 dofs, so a level's product is an M = 128 tile (levels up to 64 wide use M = 64).  One-level form
    (the oracle then needs no eigensolves), 16 right-hand sides."""
    p = W.small_problem_3d(cells=32, parts=4, k=20.0, overlap=2, seed=11)
    h = hk.setup_problem(p, precision=hk.HK_SPLIT_BF16_PRECOND, levels=hk.HK_ONE_LEVEL)
    info = hk.hk_info(h)
    assert 64 < info["max_level"] <= 128 and info["tc_record_bytes"] > 0, info["max_level"]
    o = OS.setup_problem(p, levels="one")
    v = np.random.default_rng(12).standard_normal((16, o.n))
    hk.hk_set_sweep_path(h, hk.HK_SWEEPS_TENSOR_CORE)
    z = hk.hk_apply_precond(h, v)
    hk.hk_destroy(h)
    assert np.all(_rel_rows(z, np.stack([o.precond.apply(vi) for vi in v])) <= TOL_SPLIT)
