"""The allocation-free preconditioner apply (hk_apply_precond_noalloc) gives the
same z = M^{-1} v as hk_apply_precond.

Callers that may not allocate device memory (code recording a CUDA graph, or a
framework that forbids allocations on its hot path) use this entry point: it
keeps its intermediate vectors in a fixed device array of the library.  The
test calls it through the C ABI twice in a row with different vectors, for
both precision forms, and checks each result against the allocating entry
point within the 1e-10 relative tolerance of the other apply tests.  It also
checks that a request larger than the fixed array is refused before any work.
A third test runs in a fresh process in which the allocation-free apply is
the first apply made, with subdomains large enough (about 1,200 dofs, 8
right-hand sides, FP64) that the coarse restriction needs more shared memory
than the default limit: the entry point must raise that limit itself.
This file is collected last so that a failure here leaves every other test
already run; it passes alone and after the rest.
"""
import ctypes
import os
import subprocess
import sys
import textwrap

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


ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _big_problem():
    # h = 1/128, 4 x 4 boxes: subdomains of up to 35^2 = 1,225 dofs
    return W.small_problem(cells=128, parts=4, k=20.0, overlap=2, checker=4, seed=12)


def test_noalloc_as_the_first_apply_of_a_process(tmp_path):
    from oracle import solver as OS
    out = tmp_path / "z.npy"
    code = textwrap.dedent(f"""
        import sys
        sys.path.insert(0, {ROOT!r})
        sys.path.insert(0, {os.path.join(ROOT, "tests")!r})
        import numpy as np, torch
        from paper_2406_06283_gb300 import hk
        from test_zz_no_alloc import _big_problem
        p = _big_problem()
        h = hk.setup_problem(p, precision=hk.HK_FP64)
        info = hk.hk_info(h)
        assert info["max_dof"] > 768, info["max_dof"]
        v = np.random.default_rng(13).standard_normal((8, p.mesh.n_dofs))
        v_dev = torch.tensor(v, dtype=torch.float64, device="cuda")
        z_dev = torch.full_like(v_dev, float("nan"))
        torch.cuda.synchronize()
        st = hk.lib().hk_apply_precond_noalloc(h.ptr, 8, v_dev.data_ptr(), z_dev.data_ptr())
        assert st == hk.HK_OK, (st, hk.lib().hk_last_error())
        assert hk.hk_check_status(h) == hk.HK_OK
        torch.cuda.synchronize()
        np.save({str(out)!r}, z_dev.cpu().numpy())
        hk.hk_destroy(h)
    """)
    r = subprocess.run([sys.executable, "-c", code], capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stdout[-2000:] + r.stderr[-4000:]
    got = np.load(out)
    p = _big_problem()
    o = OS.setup_problem(p)
    v = np.random.default_rng(13).standard_normal((8, p.mesh.n_dofs))
    want = np.stack([o.precond.apply(vi) for vi in v])
    assert np.all(np.isfinite(got))
    assert np.linalg.norm(got - want) <= 1e-10 * np.linalg.norm(want)
