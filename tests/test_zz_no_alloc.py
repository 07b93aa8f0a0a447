"""The allocation-free preconditioner apply (hk_apply_precond_noalloc) gives the
same z = M^{-1} v as hk_apply_precond.

Callers that may not allocate device memory (code recording a CUDA graph, or a
framework that forbids allocations on its hot path) use this entry point: it
keeps its intermediate vectors in a fixed device array of the library.  The
test calls it through the C ABI twice in a row with different vectors, for
both precision forms, and checks each result against the allocating entry
point within the 1e-10 relative tolerance of the other apply tests.  It also
checks that a request larger than the fixed array is refused before any work.
This file is collected last so that a failure here leaves every other test
already run; it passes alone and after the rest.
"""
import ctypes

import numpy as np
import pytest

from paper_2406_06283_gb300 import hk
from paper_2406_06283_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _noalloc(h, v_dev, z_dev, n_rhs=None):
    L = hk.lib()
    L.hk_apply_precond_noalloc.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_void_p, ctypes.c_void_p]
    L.hk_apply_precond_noalloc.restype = ctypes.c_int
    s = int(v_dev.shape[0]) if n_rhs is None else n_rhs
    return L.hk_apply_precond_noalloc(h.ptr, s, ctypes.c_void_p(v_dev.data_ptr()), ctypes.c_void_p(z_dev.data_ptr()))


@pytest.mark.parametrize("precision", [hk.HK_FP64, hk.HK_FP32_PRECOND])
def test_noalloc_apply_matches_allocating_apply(precision):
    import torch
    p = W.small_problem(cells=24, parts=3, k=12.0, overlap=2, checker=3, seed=8)
    h = hk.setup_problem(p, precision=precision)
    rng = np.random.default_rng(11)
    for call in range(2):
        v = rng.standard_normal((2, p.mesh.n_dofs))
        want = hk.hk_apply_precond(h, v)
        v_dev = torch.tensor(v, dtype=torch.float64, device="cuda")
        z_dev = torch.full_like(v_dev, float("nan"))
        torch.cuda.synchronize()
        assert _noalloc(h, v_dev, z_dev) == hk.HK_OK, hk.lib().hk_last_error()
        torch.cuda.synchronize()
        got = z_dev.cpu().numpy()
        assert np.all(np.isfinite(got)), f"call {call}"
        assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want), f"call {call}"
    hk.hk_destroy(h)


def test_noalloc_refuses_requests_beyond_its_array():
    import torch
    p = W.small_problem(cells=24, parts=3, k=12.0, overlap=2, checker=3, seed=8)
    h = hk.setup_problem(p)
    v_dev = torch.zeros((1, p.mesh.n_dofs), dtype=torch.float64, device="cuda")
    z_dev = torch.zeros_like(v_dev)
    # far more right-hand sides than 8 MiB can hold: refused before any launch or access
    assert _noalloc(h, v_dev, z_dev, n_rhs=100000) == hk.HK_UNSUPPORTED
    assert b"scratch" in hk.lib().hk_last_error()
    hk.hk_destroy(h)
