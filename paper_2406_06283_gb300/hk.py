"""Thin ctypes binding of libhkgeneo.so (declared in include/hkgeneo.h).

Argument marshalling only: every step of setup and solve runs in the
library's CUDA kernels.  Functions carry the C names (hk_setup, hk_solve,
...).  Host arrays are numpy; device arrays are torch CUDA tensors (used only
for their memory).  A missing library raises HKLibraryMissing - there is no
fallback path.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass

import numpy as np

_PKG = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_PKG, "_lib", "libhkgeneo.so")

HK_OK, HK_BAD_ARG, HK_SINGULAR_LOCAL, HK_SINGULAR_COARSE, HK_EIG_FAIL = 0, 1, 2, 3, 4
HK_NO_CONVERGENCE, HK_OOM, HK_TIMEOUT, HK_CUDA_ERROR, HK_UNSUPPORTED, HK_PENDING = 5, 6, 7, 8, 9, 10
HK_FP64, HK_FP32_PRECOND, HK_SPLIT_BF16_PRECOND = 0, 1, 2
HK_SWEEPS_AUTO, HK_SWEEPS_CUDA_CORE, HK_SWEEPS_TENSOR_CORE = 0, 1, 2
HK_TWO_LEVEL, HK_ONE_LEVEL, HK_COARSE_ONLY = 0, 1, 2
HK_AS, HK_RAS_POU = 0, 1


class HKLibraryMissing(RuntimeError):
    pass


class HKError(RuntimeError):
    def __init__(self, status: int, where: str, msg: str):
        super().__init__(f"{where}: status {status} ({_status_name(status)}): {msg}")
        self.status = status


class hk_mesh(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int), ("xyz", C.POINTER(C.c_double)),
                ("n_elems", C.c_int), ("elems", C.POINTER(C.c_int32)), ("is_boundary", C.POINTER(C.c_uint8))]


class hk_params(C.Structure):
    _fields_ = [("n_sub", C.c_int), ("elem_to_sub", C.POINTER(C.c_int32)), ("overlap_layers", C.c_int),
                ("tau", C.c_double), ("precision", C.c_int), ("levels", C.c_int), ("weighting", C.c_int),
                ("restart", C.c_int), ("max_iters", C.c_int)]


class hk_info_t(C.Structure):
    _fields_ = [("dim", C.c_int), ("n_nodes", C.c_int), ("n_elems", C.c_int), ("n_dofs", C.c_int),
                ("n_sub", C.c_int), ("n0", C.c_int), ("max_mu", C.c_int), ("lambda_elems", C.c_int),
                ("max_level", C.c_int), ("max_dof", C.c_int), ("nnz", C.c_int), ("precision", C.c_int),
                ("levels", C.c_int), ("bytes_resident", C.c_size_t), ("factor_elems", C.c_longlong),
                ("dof_total", C.c_longlong), ("coarse_elems", C.c_longlong), ("lower_nnz", C.c_longlong),
                ("setup_ms", C.c_double * 8), ("bytes_peak", C.c_size_t), ("graph_solves", C.c_longlong),
                ("eigen_kernel_ms", C.c_double * 4), ("eigen_kernel_gflop", C.c_double * 4),
                ("tc_record_bytes", C.c_longlong), ("last_sweeps", C.c_int), ("twist_moved", C.c_int),
                ("local_growth", C.c_double * 2), ("fine_subdomains", C.c_int), ("fine_lambda_elems", C.c_int),
                ("fine_max_dof", C.c_int), ("fine_dof_total", C.c_longlong), ("levels_merged", C.c_int)]


class hk_theory_t(C.Structure):
    _fields_ = [("Lambda", C.c_double), ("tau", C.c_double), ("tau_is_lower_bound", C.c_int), ("Theta", C.c_double),
                ("k", C.c_double), ("H_f", C.c_double), ("c_stab", C.c_double), ("s", C.c_double),
                ("gamma", C.c_double), ("guaranteed", C.c_int)]


class hk_request_info(C.Structure):
    _fields_ = [("submit_ms", C.c_double), ("start_ms", C.c_double), ("end_ms", C.c_double),
                ("batch_rhs", C.c_int32), ("setup_ran", C.c_int32), ("slot", C.c_int32), ("n_rhs", C.c_int32)]


class hk_server_stats(C.Structure):
    _fields_ = [("submitted", C.c_longlong), ("completed", C.c_longlong), ("failed", C.c_longlong),
                ("setups", C.c_longlong), ("evictions", C.c_longlong), ("batches", C.c_longlong),
                ("cache_hits", C.c_longlong), ("resident_ops", C.c_int), ("n_ops", C.c_int), ("queued", C.c_int),
                ("bytes_in_use", C.c_size_t), ("bytes_peak", C.c_size_t), ("budget", C.c_size_t)]


_lib = None
_P = C.c_void_p


def lib():
    """Loads libhkgeneo.so once; raises HKLibraryMissing if it was not built."""
    global _lib
    if _lib is not None:
        return _lib
    if not os.path.exists(LIB_PATH):
        raise HKLibraryMissing(f"{LIB_PATH} not found: run `python -m paper_2406_06283_gb300.build`")
    L = C.CDLL(LIB_PATH)
    L.hk_setup.argtypes = [C.POINTER(hk_mesh), _P, C.c_double, C.POINTER(hk_params), _P, C.POINTER(_P)]
    L.hk_setup_device.argtypes = [C.POINTER(hk_mesh), _P, C.c_double, C.POINTER(hk_params), _P, C.POINTER(_P)]
    L.hk_setup_nested.argtypes = [C.POINTER(hk_mesh), _P, C.c_double, C.POINTER(hk_params), C.c_int, _P, C.c_int, _P,
                                  C.POINTER(_P)]
    L.hk_setup_nested_device.argtypes = [C.POINTER(hk_mesh), _P, C.c_double, C.POINTER(hk_params), C.c_int, _P,
                                         C.c_int, _P, C.POINTER(_P)]
    L.hk_set_timing.argtypes = [_P, C.c_int]
    L.hk_set_solve_graphs.argtypes = [_P, C.c_int]
    L.hk_set_solve_graphs.restype = C.c_int
    L.hk_kernel_times.argtypes = [_P, _P, _P]
    L.hk_kernel_launches.argtypes = []
    L.hk_kernel_launches.restype = C.c_longlong
    L.hk_solve.argtypes = [_P, C.c_int, _P, C.c_double, _P, _P, _P, _P]
    L.hk_solve_device.argtypes = [_P, C.c_int, _P, C.c_double, _P, _P, _P, _P]
    L.hk_info.argtypes = [_P, C.POINTER(hk_info_t)]
    L.hk_destroy.argtypes = [_P]
    L.hk_status_string.argtypes = [C.c_int]
    L.hk_status_string.restype = C.c_char_p
    L.hk_last_error.restype = C.c_char_p
    L.hk_get_matrix.argtypes = [_P, C.c_int, _P, _P, _P]
    L.hk_get_subdomain.argtypes = [_P, C.c_int, _P, _P, _P, _P]
    L.hk_get_mu.argtypes = [_P, _P]
    L.hk_get_eigen.argtypes = [_P, C.c_int, _P, _P]
    L.hk_get_coarse.argtypes = [_P, _P, _P]
    L.hk_apply_precond.argtypes = [_P, C.c_int, _P, _P]
    L.hk_matvec.argtypes = [_P, C.c_int, _P, _P]
    L.hk_assemble_load.argtypes = [_P, _P, _P]
    L.hk_server_create.argtypes = [C.c_size_t, C.c_int, C.c_int, C.POINTER(_P)]
    L.hk_server_add_operator.argtypes = [_P, C.POINTER(hk_mesh), _P, C.c_double, C.POINTER(hk_params),
                                         C.POINTER(C.c_uint64)]
    L.hk_server_submit.argtypes = [_P, C.c_uint64, C.c_int, _P, C.c_double, C.POINTER(C.c_uint64)]
    L.hk_server_poll.argtypes = [_P, C.c_uint64, C.c_int, _P, _P, _P, _P, C.POINTER(hk_request_info)]
    L.hk_server_get_stats.argtypes = [_P, C.POINTER(hk_server_stats)]
    L.hk_server_destroy.argtypes = [_P]
    L.hk_check_status.argtypes = [_P]
    L.hk_set_wait_limit.argtypes = [_P, C.c_int]
    L.hk_apply_precond_noalloc.argtypes = [_P, C.c_int, _P, _P]
    L.hk_set_sweep_path.argtypes = [_P, C.c_int]
    L.hk_solve_left_dk.argtypes = [_P, C.c_int, _P, C.c_double, _P, _P, _P, _P, _P]
    L.hk_solve_left_dk_device.argtypes = [_P, C.c_int, _P, C.c_double, _P, _P, _P, _P, _P]
    L.hk_theory.argtypes = [_P, C.c_double, C.c_double, C.POINTER(hk_theory_t)]
    for f in ("hk_server_create", "hk_server_add_operator", "hk_server_submit", "hk_server_poll",
              "hk_server_get_stats", "hk_server_destroy"):
        getattr(L, f).restype = C.c_int
    for f in ("hk_setup", "hk_setup_device", "hk_set_timing", "hk_kernel_times", "hk_solve", "hk_solve_device", "hk_info", "hk_destroy", "hk_get_matrix",
              "hk_get_subdomain", "hk_get_mu", "hk_get_eigen", "hk_get_coarse", "hk_apply_precond", "hk_matvec",
              "hk_assemble_load", "hk_check_status", "hk_set_wait_limit", "hk_apply_precond_noalloc",
              "hk_set_sweep_path", "hk_solve_left_dk", "hk_solve_left_dk_device", "hk_theory", "hk_setup_nested",
              "hk_setup_nested_device"):
        getattr(L, f).restype = C.c_int
    _lib = L
    return L


def _status_name(s: int) -> str:
    try:
        return lib().hk_status_string(s).decode()
    except Exception:  # noqa: BLE001
        return str(s)


def _check(status: int, where: str, ok=(HK_OK,)):
    if status not in ok:
        raise HKError(status, where, lib().hk_last_error().decode())
    return status


def _ptr(a: np.ndarray):
    return a.ctypes.data_as(_P)


@dataclass
class Handle:
    ptr: C.c_void_p
    n: int
    max_iters: int
    _keep: tuple = ()

    def __del__(self):
        try:
            hk_destroy(self)
        except Exception:  # noqa: BLE001
            pass


def hk_setup(xyz, elems, is_boundary, elem_coeff, k, elem_to_sub, n_sub, overlap=2, tau=0.5,
             precision=HK_FP64, levels=HK_TWO_LEVEL, weighting=HK_AS, restart=50, max_iters=1000,
             stream=None) -> Handle:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    bnd = np.ascontiguousarray(is_boundary, dtype=np.uint8)
    coeff = np.ascontiguousarray(elem_coeff, dtype=np.float64)
    e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
    mesh = hk_mesh(xyz.shape[1], xyz.shape[0], xyz.ctypes.data_as(C.POINTER(C.c_double)), elems.shape[0],
                   elems.ctypes.data_as(C.POINTER(C.c_int32)), bnd.ctypes.data_as(C.POINTER(C.c_uint8)))
    prm = hk_params(int(n_sub), e2s.ctypes.data_as(C.POINTER(C.c_int32)), int(overlap), float(tau), int(precision),
                    int(levels), int(weighting), int(restart), int(max_iters))
    out = _P()
    _check(lib().hk_setup(C.byref(mesh), _ptr(coeff), float(k), C.byref(prm), _P(stream or 0), C.byref(out)),
           "hk_setup")
    h = Handle(out, int((bnd == 0).sum()), int(max_iters))
    return h


def hk_setup_nested(xyz, elems, is_boundary, elem_coeff, k, elem_to_sub, n_sub, elem_to_fine, n_fine_labels,
                    overlap=2, fine_overlap=1, tau=0.5, precision=HK_FP64, weighting=HK_AS, restart=50,
                    max_iters=1000, stream=None) -> Handle:
    """The nested coarse/fine decompositions of Sec. 2.3 (hk_setup_nested)."""
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    bnd = np.ascontiguousarray(is_boundary, dtype=np.uint8)
    coeff = np.ascontiguousarray(elem_coeff, dtype=np.float64)
    e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
    e2f = np.ascontiguousarray(elem_to_fine, dtype=np.int32)
    mesh = hk_mesh(xyz.shape[1], xyz.shape[0], xyz.ctypes.data_as(C.POINTER(C.c_double)), elems.shape[0],
                   elems.ctypes.data_as(C.POINTER(C.c_int32)), bnd.ctypes.data_as(C.POINTER(C.c_uint8)))
    prm = hk_params(int(n_sub), e2s.ctypes.data_as(C.POINTER(C.c_int32)), int(overlap), float(tau), int(precision),
                    HK_TWO_LEVEL, int(weighting), int(restart), int(max_iters))
    out = _P()
    _check(lib().hk_setup_nested(C.byref(mesh), _ptr(coeff), float(k), C.byref(prm), int(n_fine_labels), _ptr(e2f),
                                 int(fine_overlap), _P(stream or 0), C.byref(out)), "hk_setup_nested")
    return Handle(out, int((bnd == 0).sum()), int(max_iters))


def setup_problem_nested(p, elem_to_fine, n_fine_labels, fine_overlap=1, precision=HK_FP64, weighting=HK_AS,
                         stream=None) -> Handle:
    """hk_setup_nested for a workloads.Problem and a fine element labelling."""
    m = p.mesh
    return hk_setup_nested(m.xyz, m.elems, m.is_boundary, p.coeff, p.k, p.elem_to_sub, p.n_sub, elem_to_fine,
                           n_fine_labels, p.overlap, fine_overlap, p.tau, precision, weighting, p.restart,
                           p.max_iters, stream)


def hk_setup_device(xyz_dev, elems_dev, is_boundary_dev, elem_coeff_dev, k, elem_to_sub_dev, n_sub, overlap=2,
                    tau=0.5, precision=HK_FP64, levels=HK_TWO_LEVEL, weighting=HK_AS, restart=50, max_iters=1000,
                    stream=None, n_dofs=None) -> Handle:
    """Setup from device-resident torch tensors (float64 xyz (n_nodes, dim), int32 elems, uint8 flags,
    float64 coefficients, int32 partition)."""
    mesh = hk_mesh(int(xyz_dev.shape[1]), int(xyz_dev.shape[0]), C.cast(_P(xyz_dev.data_ptr()), C.POINTER(C.c_double)),
                   int(elems_dev.shape[0]), C.cast(_P(elems_dev.data_ptr()), C.POINTER(C.c_int32)),
                   C.cast(_P(is_boundary_dev.data_ptr()), C.POINTER(C.c_uint8)))
    prm = hk_params(int(n_sub), C.cast(_P(elem_to_sub_dev.data_ptr()), C.POINTER(C.c_int32)), int(overlap), float(tau),
                    int(precision), int(levels), int(weighting), int(restart), int(max_iters))
    out = _P()
    _check(lib().hk_setup_device(C.byref(mesh), _P(elem_coeff_dev.data_ptr()), float(k), C.byref(prm),
                                 _P(stream or 0), C.byref(out)), "hk_setup_device")
    n = n_dofs if n_dofs is not None else int((is_boundary_dev == 0).sum().item())
    return Handle(out, n, int(max_iters))


def hk_setup_nested_device(xyz_dev, elems_dev, is_boundary_dev, elem_coeff_dev, k, elem_to_sub_dev, n_sub,
                           elem_to_fine_dev, n_fine_labels, overlap=2, fine_overlap=1, tau=0.5, precision=HK_FP64,
                           weighting=HK_AS, restart=50, max_iters=1000, stream=None, n_dofs=None) -> Handle:
    """hk_setup_nested_device from device-resident torch tensors (as hk_setup_device, plus int32 fine labels)."""
    mesh = hk_mesh(int(xyz_dev.shape[1]), int(xyz_dev.shape[0]), C.cast(_P(xyz_dev.data_ptr()), C.POINTER(C.c_double)),
                   int(elems_dev.shape[0]), C.cast(_P(elems_dev.data_ptr()), C.POINTER(C.c_int32)),
                   C.cast(_P(is_boundary_dev.data_ptr()), C.POINTER(C.c_uint8)))
    prm = hk_params(int(n_sub), C.cast(_P(elem_to_sub_dev.data_ptr()), C.POINTER(C.c_int32)), int(overlap), float(tau),
                    int(precision), HK_TWO_LEVEL, int(weighting), int(restart), int(max_iters))
    out = _P()
    _check(lib().hk_setup_nested_device(C.byref(mesh), _P(elem_coeff_dev.data_ptr()), float(k), C.byref(prm),
                                        int(n_fine_labels), _P(elem_to_fine_dev.data_ptr()), int(fine_overlap),
                                        _P(stream or 0), C.byref(out)), "hk_setup_nested_device")
    n = n_dofs if n_dofs is not None else int((is_boundary_dev == 0).sum().item())
    return Handle(out, n, int(max_iters))


HK_T_NAMES = ("local_apply", "coarse_solve", "scatter", "spmv", "arnoldi", "cycle_end")


def hk_kernel_launches() -> int:
    """Kernels the library has launched in this process so far."""
    return int(lib().hk_kernel_launches())


def hk_set_solve_graphs(h: Handle, on: bool = True):
    _check(lib().hk_set_solve_graphs(h.ptr, int(bool(on))), "hk_set_solve_graphs")


def hk_set_sweep_path(h: Handle, path: int):
    """Local sweeps of the split-BF16 form: HK_SWEEPS_AUTO, HK_SWEEPS_CUDA_CORE or HK_SWEEPS_TENSOR_CORE."""
    _check(lib().hk_set_sweep_path(h.ptr, int(path)), "hk_set_sweep_path")


def hk_check_status(h: Handle) -> int:
    """Status of the handle's device work since the last check (the record is cleared)."""
    return int(lib().hk_check_status(h.ptr))


def hk_set_wait_limit(h: Handle, polls: int):
    """Test hook: polls of the cooperative Gram-Schmidt grid barrier before it gives up (0 = default)."""
    _check(lib().hk_set_wait_limit(h.ptr, int(polls)), "hk_set_wait_limit")


def hk_set_timing(h: Handle, on: bool = True):
    _check(lib().hk_set_timing(h.ptr, int(bool(on))), "hk_set_timing")


def hk_kernel_times(h: Handle) -> dict:
    ms = np.zeros(len(HK_T_NAMES))
    cnt = np.zeros(len(HK_T_NAMES), dtype=np.int32)
    _check(lib().hk_kernel_times(h.ptr, _ptr(ms), _ptr(cnt)), "hk_kernel_times")
    return {n: (float(ms[i]), int(cnt[i])) for i, n in enumerate(HK_T_NAMES)}


def setup_problem(p, precision=HK_FP64, levels=HK_TWO_LEVEL, weighting=HK_AS, stream=None) -> Handle:
    """hk_setup for a workloads.Problem."""
    m = p.mesh
    return hk_setup(m.xyz, m.elems, m.is_boundary, p.coeff, p.k, p.elem_to_sub, p.n_sub, p.overlap, p.tau,
                    precision, levels, weighting, p.restart, p.max_iters, stream)


def hk_destroy(h: Handle):
    if h.ptr is not None and h.ptr.value:
        lib().hk_destroy(h.ptr)
        h.ptr = _P()


@dataclass
class SolveResult:
    u: object            # (n_rhs, n) numpy array, or a torch tensor for hk_solve_device
    iters: np.ndarray
    history: np.ndarray  # (n_rhs, max_iters); entries past iters[r] are zero
    true_rel_res: np.ndarray
    status: int


def hk_solve(h: Handle, rhs, tol=1e-8) -> SolveResult:
    rhs = np.ascontiguousarray(np.atleast_2d(rhs), dtype=np.float64)
    s = rhs.shape[0]
    u = np.zeros_like(rhs)
    it = np.zeros(s, dtype=np.int32)
    hist = np.zeros((s, h.max_iters))
    res = np.zeros(s)
    st = _check(lib().hk_solve(h.ptr, s, _ptr(rhs), float(tol), _ptr(u), _ptr(it), _ptr(hist), _ptr(res)),
                "hk_solve", ok=(HK_OK, HK_NO_CONVERGENCE))
    return SolveResult(u, it, hist, res, st)


def hk_solve_left_dk(h: Handle, rhs, tol=1e-8):
    """Left-preconditioned GMRES in the D_k inner product (Thm. 3.1).  Returns (SolveResult, pc_rel_res):
    the history holds ||M^{-1} r_j||_D / ||M^{-1} f||_D, true_rel_res ||f - B u|| / ||f||."""
    rhs = np.ascontiguousarray(np.atleast_2d(rhs), dtype=np.float64)
    s = rhs.shape[0]
    u = np.zeros_like(rhs)
    it = np.zeros(s, dtype=np.int32)
    hist = np.zeros((s, h.max_iters))
    res = np.zeros(s)
    pc = np.zeros(s)
    st = _check(lib().hk_solve_left_dk(h.ptr, s, _ptr(rhs), float(tol), _ptr(u), _ptr(it), _ptr(hist), _ptr(res),
                                       _ptr(pc)), "hk_solve_left_dk", ok=(HK_OK, HK_NO_CONVERGENCE))
    return SolveResult(u, it, hist, res, st), pc


def hk_solve_left_dk_device(h: Handle, rhs_dev, u_dev, tol=1e-8):
    """rhs_dev, u_dev: contiguous float64 CUDA tensors of shape (n_rhs, n).  Returns (iters, true, pc)."""
    s = int(rhs_dev.shape[0])
    it = np.zeros(s, dtype=np.int32)
    res = np.zeros(s)
    pc = np.zeros(s)
    _check(lib().hk_solve_left_dk_device(h.ptr, s, _P(rhs_dev.data_ptr()), float(tol), _P(u_dev.data_ptr()),
                                         _ptr(it), None, _ptr(res), _ptr(pc)),
           "hk_solve_left_dk_device", ok=(HK_OK, HK_NO_CONVERGENCE))
    return it, res, pc


def hk_theory(h: Handle, c_stab: float, H_f: float = 0.0) -> dict:
    """Lambda, tau, Theta, s, gamma of Thm. 3.1 (H_f <= 0: the largest subdomain bounding-box diagonal)."""
    t = hk_theory_t()
    _check(lib().hk_theory(h.ptr, float(c_stab), float(H_f), C.byref(t)), "hk_theory")
    return {f: getattr(t, f) for f, _ in hk_theory_t._fields_}


def hk_solve_device(h: Handle, rhs_dev, u_dev, tol=1e-8, history=False) -> SolveResult:
    """rhs_dev, u_dev: contiguous float64 CUDA tensors of shape (n_rhs, n)."""
    s = int(rhs_dev.shape[0])
    it = np.zeros(s, dtype=np.int32)
    hist = np.zeros((s, h.max_iters)) if history else None
    res = np.zeros(s)
    st = _check(lib().hk_solve_device(h.ptr, s, _P(rhs_dev.data_ptr()), float(tol), _P(u_dev.data_ptr()), _ptr(it),
                                      _ptr(hist) if history else None, _ptr(res)),
                "hk_solve_device", ok=(HK_OK, HK_NO_CONVERGENCE))
    return SolveResult(u_dev, it, hist, res, st)


def hk_info(h: Handle) -> dict:
    info = hk_info_t()
    _check(lib().hk_info(h.ptr, C.byref(info)), "hk_info")
    d = {f: getattr(info, f) for f, _ in hk_info_t._fields_
         if f not in ("setup_ms", "eigen_kernel_ms", "eigen_kernel_gflop", "local_growth")}
    d["local_growth"] = list(info.local_growth)
    d["setup_ms"] = list(info.setup_ms)
    d["eigen_kernel_ms"] = list(info.eigen_kernel_ms)
    d["eigen_kernel_gflop"] = list(info.eigen_kernel_gflop)
    return d


def hk_get_matrix(h: Handle, which=0):
    inf = hk_info(h)
    n, nnz = inf["n_dofs"], inf["nnz"]
    rp = np.zeros(n + 1, dtype=np.int32)
    col = np.zeros(nnz, dtype=np.int32)
    val = np.zeros(nnz)
    _check(lib().hk_get_matrix(h.ptr, int(which), _ptr(rp), _ptr(col), _ptr(val)), "hk_get_matrix")
    return rp, col, val


def hk_get_subdomain(h: Handle, i: int) -> dict:
    sizes = np.zeros(4, dtype=np.int32)
    _check(lib().hk_get_subdomain(h.ptr, int(i), _ptr(sizes), None, None, None), "hk_get_subdomain")
    nI, nG, L, m = (int(x) for x in sizes)
    dof = np.zeros(nI, dtype=np.int32)
    gam = np.zeros(max(nG, 1), dtype=np.int32)
    lp = np.zeros(L + 1, dtype=np.int32)
    _check(lib().hk_get_subdomain(h.ptr, int(i), _ptr(sizes), _ptr(dof), _ptr(gam), _ptr(lp)), "hk_get_subdomain")
    return {"dof": dof, "gamma": gam[:nG], "level_ptr": lp, "m": m}


def hk_get_mu(h: Handle) -> np.ndarray:
    mu = np.zeros(h.n, dtype=np.int32)
    _check(lib().hk_get_mu(h.ptr, _ptr(mu)), "hk_get_mu")
    return mu


def hk_get_eigen(h: Handle, i: int):
    sd = hk_get_subdomain(h, i)
    m, nI = sd["m"], sd["dof"].size
    lam = np.zeros(max(m, 1))
    Z = np.zeros((nI, max(m, 1)))
    _check(lib().hk_get_eigen(h.ptr, int(i), _ptr(lam), _ptr(Z)), "hk_get_eigen")
    return lam[:m], Z[:, :m], sd["dof"]


def hk_get_coarse(h: Handle):
    n0 = hk_info(h)["n0"]
    E = np.zeros((n0, n0))
    Ei = np.zeros((n0, n0))
    _check(lib().hk_get_coarse(h.ptr, _ptr(E), _ptr(Ei)), "hk_get_coarse")
    return E, Ei


def hk_apply_precond(h: Handle, v) -> np.ndarray:
    v = np.ascontiguousarray(np.atleast_2d(v), dtype=np.float64)
    z = np.zeros_like(v)
    _check(lib().hk_apply_precond(h.ptr, v.shape[0], _ptr(v), _ptr(z)), "hk_apply_precond")
    return z


def hk_matvec(h: Handle, x) -> np.ndarray:
    x = np.ascontiguousarray(np.atleast_2d(x), dtype=np.float64)
    y = np.zeros_like(x)
    _check(lib().hk_matvec(h.ptr, x.shape[0], _ptr(x), _ptr(y)), "hk_matvec")
    return y


def hk_assemble_load(h: Handle, f_nodal) -> np.ndarray:
    f = np.ascontiguousarray(f_nodal, dtype=np.float64)
    out = np.zeros(h.n)
    _check(lib().hk_assemble_load(h.ptr, _ptr(f), _ptr(out)), "hk_assemble_load")
    return out


# ---- serving (hk_server_*) ----

@dataclass
class Server:
    ptr: C.c_void_p
    n_dofs: dict        # op id -> n_dofs
    max_iters: dict     # op id -> max_iters

    def __del__(self):
        try:
            hk_server_destroy(self)
        except Exception:  # noqa: BLE001
            pass


def hk_server_create(budget_bytes: int, n_slots: int = 4, max_batch_rhs: int = 16) -> Server:
    out = _P()
    _check(lib().hk_server_create(int(budget_bytes), int(n_slots), int(max_batch_rhs), C.byref(out)),
           "hk_server_create")
    return Server(out, {}, {})


def hk_server_add_operator(srv: Server, xyz, elems, is_boundary, elem_coeff, k, elem_to_sub, n_sub, overlap=2,
                           tau=0.5, precision=HK_FP64, levels=HK_TWO_LEVEL, weighting=HK_AS, restart=50,
                           max_iters=1000) -> int:
    xyz = np.ascontiguousarray(xyz, dtype=np.float64)
    elems = np.ascontiguousarray(elems, dtype=np.int32)
    bnd = np.ascontiguousarray(is_boundary, dtype=np.uint8)
    coeff = np.ascontiguousarray(elem_coeff, dtype=np.float64)
    e2s = np.ascontiguousarray(elem_to_sub, dtype=np.int32)
    mesh = hk_mesh(xyz.shape[1], xyz.shape[0], xyz.ctypes.data_as(C.POINTER(C.c_double)), elems.shape[0],
                   elems.ctypes.data_as(C.POINTER(C.c_int32)), bnd.ctypes.data_as(C.POINTER(C.c_uint8)))
    prm = hk_params(int(n_sub), e2s.ctypes.data_as(C.POINTER(C.c_int32)), int(overlap), float(tau), int(precision),
                    int(levels), int(weighting), int(restart), int(max_iters))
    op = C.c_uint64()
    _check(lib().hk_server_add_operator(srv.ptr, C.byref(mesh), _ptr(coeff), float(k), C.byref(prm), C.byref(op)),
           "hk_server_add_operator")
    srv.n_dofs[op.value] = int((bnd == 0).sum())
    srv.max_iters[op.value] = int(max_iters)
    return op.value


def server_add_problem(srv: Server, p, precision=HK_FP64) -> int:
    """hk_server_add_operator for a workloads.Problem."""
    m = p.mesh
    return hk_server_add_operator(srv, m.xyz, m.elems, m.is_boundary, p.coeff, p.k, p.elem_to_sub, p.n_sub,
                                  p.overlap, p.tau, precision, HK_TWO_LEVEL, HK_AS, p.restart, p.max_iters)


def hk_server_submit(srv: Server, op: int, rhs, tol=1e-8) -> int:
    rhs = np.ascontiguousarray(np.atleast_2d(rhs), dtype=np.float64)
    t = C.c_uint64()
    _check(lib().hk_server_submit(srv.ptr, C.c_uint64(op), rhs.shape[0], _ptr(rhs), float(tol), C.byref(t)),
           "hk_server_submit")
    return t.value


@dataclass
class ServedResult:
    u: np.ndarray
    iters: np.ndarray
    history: np.ndarray
    true_rel_res: np.ndarray
    status: int
    info: dict


def hk_server_poll(srv: Server, ticket: int, op: int, n_rhs: int, wait_ms: int = -1, raise_on_failure: bool = True):
    """None while the request runs; else a ServedResult.  A failed request raises HKError, or with
    raise_on_failure=False comes back as a ServedResult whose status is the failure's."""
    n, mi = srv.n_dofs[op], srv.max_iters[op]
    u = np.zeros((n_rhs, n))
    it = np.zeros(n_rhs, dtype=np.int32)
    hist = np.zeros((n_rhs, mi))
    res = np.zeros(n_rhs)
    info = hk_request_info()
    st = lib().hk_server_poll(srv.ptr, C.c_uint64(ticket), int(wait_ms), _ptr(u), _ptr(it), _ptr(hist), _ptr(res),
                              C.byref(info))
    if st == HK_PENDING:
        return None
    if raise_on_failure or st == HK_BAD_ARG:
        _check(st, "hk_server_poll", ok=(HK_OK, HK_NO_CONVERGENCE))
    return ServedResult(u, it, hist, res, st, {f: getattr(info, f) for f, _ in hk_request_info._fields_})


def hk_server_get_stats(srv: Server) -> dict:
    s = hk_server_stats()
    _check(lib().hk_server_get_stats(srv.ptr, C.byref(s)), "hk_server_get_stats")
    return {f: getattr(s, f) for f, _ in hk_server_stats._fields_}


def hk_server_destroy(srv: Server):
    if srv.ptr is not None and srv.ptr.value:
        lib().hk_server_destroy(srv.ptr)
        srv.ptr = _P()
