#!/usr/bin/env python
"""Benchmark of the two-level Schwarz / H_k-GenEO / FGMRES Helmholtz solver.

One step = one pass of the whole method over one synthetic instance: device
setup (assembly, decomposition, local factors, H_k-GenEO eigenproblems,
coarse operator) and the right-preconditioned FGMRES solve to 1e-8 relative
residual.  Default workload: 2D unit square, P1 on a '/' mesh with h = 1/256
(65,025 dofs), k = 50, 8x8 checkerboard coefficient 10^U[0,2], 8x8 box
subdomains, overlap 2, tau = 0.5, one N(0,1) right-hand side, FP32
preconditioner with FP64 Krylov.

`value` (solves/s) is measured with every input resident in HBM
(hk_setup_device + hk_solve_device); `e2e` repeats the step through the
host-pointer calls (hk_setup + hk_solve) with the copies inside the timed
region.  Between timed steps a 512 MB buffer is written to flush L2.
Under torchrun each rank solves its own replica (the method is not sharded
here): value = steps * ranks / max-over-ranks time.

--impl reference times the CPU oracle (test infrastructure, FP64 numpy/scipy)
on the same workload on this host's cores.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

from paper_2406_06283_gb300 import workloads as W  # noqa: E402

METRIC = "Helmholtz solves/s and p99 latency at 1e-8 residual; FP32-precond vs FP64 form"
PEAKS_PATH = os.path.join(ROOT, "MEASURED_PEAKS.json")
TRAFFIC_PATH = os.path.join(ROOT, "profiles", "dram_traffic.txt")
CSRC = os.path.join(ROOT, "paper_2406_06283_gb300", "csrc")
# hk_params.precision of each --precision choice (HK_FP64, HK_FP32_PRECOND, HK_SPLIT_BF16_PRECOND) and the
# arithmetic it computes in
PRECISIONS = {"fp64": 0, "fp32": 1, "split": 2}
DTYPES = {"fp64": "f64", "fp32": "f64 Krylov / f32 preconditioner",
          "split": "f64 Krylov / split-bf16 tensor-core local solves, f32 coarse"}
TC_NRHS = 16  # right-hand sides per tensor-core sweep CTA (the MMA's N)


def bf16_peak() -> float:
    try:
        with open(PEAKS_PATH) as f:
            return float(json.load(f)["bf16_tflops"])
    except Exception:  # noqa: BLE001
        return 1900.0


BF16_PEAK = bf16_peak()


def kernel_source(kernel: str) -> str | None:
    """Path of the CUDA source file whose `__global__` declaration defines `kernel` (not merely names it)."""
    import re
    pat = re.compile(rb"__global__\s+(?:void\s+)?(?:__launch_bounds__\([^)]*\)\s+)?(?:void\s+)?" +
                     re.escape(kernel.encode()) + rb"\s*\(")
    for f in sorted(os.listdir(CSRC)):
        if f.endswith(".cu") and pat.search(open(os.path.join(CSRC, f), "rb").read()):
            return os.path.join(CSRC, f)
    return None


def source_digest(kernel: str) -> str | None:
    """sha256 (first 16 hex digits) of the CUDA source file that defines `kernel`."""
    import hashlib
    path = kernel_source(kernel)
    return hashlib.sha256(open(path, "rb").read()).hexdigest()[:16] if path else None


def measured_traffic(kernel: str, workload: str):
    """DRAM bytes (read + write) per launch of `kernel` on `workload`, from the ncu record in
    profiles/dram_traffic.txt, or None when there is no record or the kernel's source file has
    changed since the counters were taken."""
    try:
        lines = open(TRAFFIC_PATH).read().splitlines()
    except OSError:
        return None
    dig = source_digest(kernel)
    for ln in lines:
        f = ln.split()
        if len(f) >= 4 and not ln.startswith("#") and f[0] == kernel and f[1] == workload:
            return int(f[3]) if f[2] == dig else None
    return None


def workload(name: str):
    if name == "c2":
        return W.config_c2()
    if name == "c1":
        return W.config_c1()
    if name == "c3":
        return W.config_c3()
    raise SystemExit(f"unknown workload {name}")


def workload_config(p, name, precision, fine_parts=0, fine_overlap=0):
    nest = (f", nested: fine {fine_parts}x{fine_parts} boxes inside the coarse subdomains, fine overlap "
            f"{fine_overlap} (Sec. 2.3)") if fine_parts else ""
    return {"workload": f"{p.name}: 2D P1 h=1/{p.mesh.cells} ({p.mesh.n_dofs} dofs), k={p.k:g}, "
                        f"{p.parts}x{p.parts} subdomains, overlap {p.overlap}, tau {p.tau}, "
                        f"FGMRES({p.restart}) to {p.tol:g}, {1 if p.rhs is None else p.rhs.shape[0]} rhs{nest}",
            "precision_form": precision, "global_batch": 1 if p.rhs is None else int(p.rhs.shape[0]),
            "l2": "flushed between timed steps (512 MB write)", "parallelism": "replicas"}


def peaks():
    try:
        with open(PEAKS_PATH) as f:
            d = json.load(f)
        return float(d["hbm_gbs"]), "measured"
    except Exception:  # noqa: BLE001
        return 6800.0, "fallback"


class ClockSampler:
    """Samples nvidia-smi clocks and throttle reasons during the timed region."""
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index: int):
        self.index = index
        self.proc = None
        self.lines = []
        self._t = None

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self._t = threading.Thread(target=self._read, daemon=True)
            self._t.start()
        except Exception:  # noqa: BLE001
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if self.proc is None:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:  # noqa: BLE001
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                mx = float(parts[2])
            except ValueError:
                continue
            for nm, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


def dist_init():
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        import torch
        import torch.distributed as dist
        backend = "nccl" if torch.cuda.is_available() else "gloo"
        dist.init_process_group(backend)
    return world, rank, local


def barrier(world):
    if world > 1:
        import torch.distributed as dist
        dist.barrier()


def max_over_ranks(x: float, world: int) -> float:
    if world == 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([x], dtype=torch.float64, device="cuda" if torch.cuda.is_available() else "cpu")
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


# ------------------------------------------------------------------ oracle arm
def oracle_step(p):
    from oracle import solver as OS
    t0 = time.perf_counter()
    h = OS.setup_problem(p)
    t1 = time.perf_counter()
    r = OS.solve(h, OS.load_vector(p), p.tol)
    t2 = time.perf_counter()
    return t1 - t0, t2 - t1, [x.iters for x in r]


class OracleSampler:
    """Bounded samples of one oracle setup + solve of a workload.  The oracle's cost separates into a
    global part (assembly, decomposition, coarse matrix and its factorisation: timed once while the
    sampler is prepared), a per-subdomain part (local pencil, eigenproblem and local LU factorisation
    of Omega_i) and a per-iteration part (one FGMRES inner step at the solve's mean Krylov depth: one
    preconditioner apply, one matvec and the modified Gram-Schmidt sweep).  A sample runs the
    per-subdomain work of one subdomain (in turn) and one inner step; the time of a whole solve is
    then  t_global + n_sub * t_subdomain + iterations * t_iteration.  With nested decompositions
    (Sec. 2.3) a sample adds one fine subdomain's LU, and the solve  n_fine * t_fine_lu  more (the
    eigenproblems stay on the coarse subdomains)."""

    def __init__(self, p, nested=None):
        import scipy.linalg as sla

        from oracle import decomposition as OD
        from oracle import fem as OF
        from oracle import geneo as OG
        from oracle import solver as OS
        self.p, self.OD, self.OF, self.OG, self.sla = p, OD, OF, OG, sla
        self.nested = nested
        t0 = time.perf_counter()
        self.h = OS.setup_problem(p, nested=nested)
        t1 = time.perf_counter()
        self.f = OS.load_vector(p)[0]
        r = OS.solve(self.h, self.f[None, :], p.tol)[0]
        t2 = time.perf_counter()
        self.iters = r.iters
        self.setup_s, self.solve_s = t1 - t0, t2 - t1
        m = p.mesh
        # global part of the setup: everything but the per-subdomain eigen and LU work
        g0 = time.perf_counter()
        OF.helmholtz_matrices(m.xyz, m.elems, p.coeff, m.is_boundary, p.k)
        OD.decompose(m.xyz, m.elems, m.is_boundary, p.elem_to_sub, p.n_sub, p.overlap)
        E = self.h.precond.E
        sla.lu_factor(E)
        self.global_s = time.perf_counter() - g0
        self.depth = max(1, min(p.restart, self.iters) // 2)
        rng = np.random.default_rng(0)
        self.V = np.linalg.qr(rng.standard_normal((self.h.n, self.depth + 1)))[0].T.copy()
        self.k = 0
        self.t_sub, self.t_it, self.t_fine = [], [], []

    def step(self):
        p, h, m = self.p, self.h, self.p.mesh
        i = self.k % p.n_sub
        self.k += 1
        t0 = time.perf_counter()
        sd = h.coarse_subs[i]
        BN, C, w = self.OG.local_pencil(m.xyz, m.elems, p.coeff, m.is_boundary, p.k, sd, h.mu_c)
        self.OG.local_eigen(BN, C, w, p.tau)
        if self.nested is None:
            Bi = h.B.tocsr()[sd.dof][:, sd.dof].toarray()
            self.sla.lu_factor(Bi)
        else:
            tf = time.perf_counter()
            fd = h.subs[(self.k - 1) % len(h.subs)]
            self.sla.lu_factor(h.B.tocsr()[fd.dof][:, fd.dof].toarray())
            self.t_fine.append(time.perf_counter() - tf)
        t1 = time.perf_counter()
        z = h.precond.apply(self.V[self.depth])
        wv = h.B @ z
        for q in range(self.depth + 1):
            wv = wv - float(np.dot(wv, self.V[q])) * self.V[q]
        np.linalg.norm(wv)
        t2 = time.perf_counter()
        self.t_sub.append(t1 - t0)
        self.t_it.append(t2 - t1)
        return t2 - t0

    def solve_seconds(self):
        t = self.global_s + self.p.n_sub * statistics.mean(self.t_sub) + self.iters * statistics.mean(self.t_it)
        if self.nested is not None:
            t += (len(self.h.subs) - self.p.n_sub) * statistics.mean(self.t_fine)
        return t

    def describe(self):
        return (f"{len(self.t_sub)} samples, each: one subdomain's local pencil + eigenproblem + LU "
                f"({1e3 * statistics.mean(self.t_sub):.0f} ms) and one FGMRES inner step at Krylov depth "
                f"{self.depth} ({1e3 * statistics.mean(self.t_it):.1f} ms); solve = global setup "
                f"{self.global_s:.2f} s + {self.p.n_sub} subdomains + {self.iters} iterations (the oracle's "
                f"count); one whole oracle setup + solve for comparison: {self.setup_s + self.solve_s:.1f} s; "
                f"numpy/scipy, BLAS threads up to {os.cpu_count()}")


def run_reference(args, world, rank):
    if rank != 0:
        return
    if args.workload in ("c4", "c5"):
        cb = serving_cpu_baseline(W.config_c5() if args.workload == "c5" else W.config_c4())
        line = {"impl": "reference", "metric": METRIC, "value": cb["value"], "unit": "solves/s",
                "n_gpus": args.gpus, "steps": 1, "warmup": 0, "ms_per_step": 1e3 / cb["value"],
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
                "data": "synthetic", "config": {"workload": f"{args.workload} operators (oracle sample)"},
                "cpu_baseline": cb,
                "e2e": {"value": cb["value"], "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return
    p = workload(args.workload)
    cores = os.cpu_count()
    smp = OracleSampler(p)
    for _ in range(args.warmup):
        smp.step()
    smp.t_sub.clear()
    smp.t_it.clear()
    step_s = [smp.step() for _ in range(args.steps)]
    s = 1 if p.rhs is None else p.rhs.shape[0]
    value = s / smp.solve_seconds()
    cb = {"value": value, "unit": "solves/s", "cores": cores, "kind": "oracle", "sample": smp.describe()}
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * statistics.mean(step_s),
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64",
            "data": "synthetic (seeded)", "config": workload_config(p, args.workload, args.precision),
            "cpu_baseline": cb,
            "e2e": {"value": value, "unit": "solves/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


def cpu_baseline(p, samples=12, nested=None):
    """The oracle as it stands on this host, timed on a bounded sample of the workload (OracleSampler)."""
    smp = OracleSampler(p, nested)
    for _ in range(samples):
        smp.step()
    s = 1 if p.rhs is None else p.rhs.shape[0]
    return {"value": s / smp.solve_seconds(), "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": smp.describe()}


# ------------------------------------------------------------------ GPU arm
def run_ours(args, world, rank, local):
    import torch

    from paper_2406_06283_gb300 import hk

    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)
    p = workload(args.workload)
    prec = PRECISIONS[args.precision]
    m = p.mesh
    rhs_host = np.ascontiguousarray(np.atleast_2d(p.rhs), dtype=np.float64)
    s = rhs_host.shape[0]
    # inputs resident in HBM
    d_xyz = torch.tensor(m.xyz, device=dev)
    d_el = torch.tensor(m.elems, dtype=torch.int32, device=dev)
    d_bnd = torch.tensor(m.is_boundary, dtype=torch.uint8, device=dev)
    d_coeff = torch.tensor(p.coeff, device=dev)
    d_e2s = torch.tensor(p.elem_to_sub, dtype=torch.int32, device=dev)
    d_rhs = torch.tensor(rhs_host, device=dev)
    d_u = torch.empty_like(d_rhs)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    sptr = stream.cuda_stream

    fine = args.fine_parts
    if fine:
        e2f_host = W.box_partition(m, fine)
        d_e2f = torch.tensor(e2f_host, dtype=torch.int32, device=dev)

    def setup_dev(precision=prec):
        if fine:  # the nested decompositions of Sec. 2.3: fine boxes inside the coarse subdomains
            return hk.hk_setup_nested_device(d_xyz, d_el, d_bnd, d_coeff, p.k, d_e2s, p.n_sub, d_e2f, fine ** m.dim,
                                             p.overlap, args.fine_overlap, p.tau, precision, hk.HK_AS, p.restart,
                                             p.max_iters, sptr, n_dofs=m.n_dofs)
        return hk.hk_setup_device(d_xyz, d_el, d_bnd, d_coeff, p.k, d_e2s, p.n_sub, p.overlap, p.tau, precision,
                                  hk.HK_TWO_LEVEL, hk.HK_AS, p.restart, p.max_iters, sptr, n_dofs=m.n_dofs)

    def device_step(record=None, timing=False, graphs=True):
        """One step: setup + solve + destroy.  With timing, the solve records per-kernel CUDA events,
        which drives its loops from the host instead of the captured graph (used once, untimed).
        graphs=False launches the solve's kernels one by one (profilers cannot see kernel nodes of a
        graph with conditional nodes)."""
        h = setup_dev()
        if not graphs:
            hk.hk_set_solve_graphs(h, False)
        if timing:
            hk.hk_set_timing(h, True)
        r = hk.hk_solve_device(h, d_rhs, d_u, p.tol)
        if record is not None:
            record.append((hk.hk_info(h), hk.hk_kernel_times(h) if timing else None, r.iters.copy()))
        hk.hk_destroy(h)
        return r

    ev = lambda: torch.cuda.Event(enable_timing=True)  # noqa: E731
    for _ in range(args.warmup):
        device_step()
    torch.cuda.synchronize()
    sampler = ClockSampler(local)
    rec = []
    step_ms = []
    if args.profile_sweeps:
        # only the local sweeps of 16 right-hand sides: tensor-core, then CUDA-core, twice each
        h = setup_dev()
        v16 = np.random.default_rng(1).standard_normal((TC_NRHS, m.n_dofs))
        for path in (hk.HK_SWEEPS_TENSOR_CORE, hk.HK_SWEEPS_CUDA_CORE):
            hk.hk_set_sweep_path(h, path)
            for _ in range(2):
                hk.hk_apply_precond(h, v16)
        hk.hk_destroy(h)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_sweeps": True, "workload": p.name}), flush=True)
        return
    if args.profile_run:
        device_step(graphs=False)
        if prec == PRECISIONS["split"]:
            # the local sweeps of 16 right-hand sides on both paths, twice each
            h = setup_dev()
            v16 = np.random.default_rng(1).standard_normal((TC_NRHS, m.n_dofs))
            for path in (hk.HK_SWEEPS_TENSOR_CORE, hk.HK_SWEEPS_CUDA_CORE):
                if path == hk.HK_SWEEPS_TENSOR_CORE and hk.hk_info(h)["tc_record_bytes"] == 0:
                    continue
                hk.hk_set_sweep_path(h, path)
                for _ in range(2):
                    hk.hk_apply_precond(h, v16)
            hk.hk_destroy(h)
        torch.cuda.synchronize()
        if rank == 0:
            print(json.dumps({"profile_run": True, "workload": p.name}), flush=True)
        return
    barrier(world)
    torch.cuda.synchronize()
    launches0 = hk.hk_kernel_launches()
    sampler.start()
    wall0 = time.perf_counter()
    for _ in range(args.steps):
        flush.fill_(1.0)
        e0, e1 = ev(), ev()
        e0.record(stream)
        device_step(rec)
        e1.record(stream)
        e1.synchronize()
        step_ms.append(e0.elapsed_time(e1))
    torch.cuda.synchronize()
    wall = time.perf_counter() - wall0
    launches = hk.hk_kernel_launches() - launches0
    barrier(world)
    clocks = sampler.stop()
    rec_t = []
    device_step(rec_t, timing=True)  # per-kernel solve timings, outside the timed region
    t_rank = sum(step_ms) / 1e3
    t_max = max_over_ranks(t_rank, world)
    value = args.steps * s * world / t_max

    # ---- e2e through the host-pointer calls (copies inside the timed region)
    h2d = m.xyz.nbytes + m.elems.astype(np.int32).nbytes + m.is_boundary.nbytes + p.coeff.nbytes + \
        p.elem_to_sub.astype(np.int32).nbytes + rhs_host.nbytes + (4 * m.n_elems if fine else 0)
    d2h = rhs_host.nbytes + 4 * s + 8 * s
    e2e_ms = []
    for k in range(max(1, min(args.steps, 5))):
        flush.fill_(1.0)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        if fine:  # the same nested decompositions as the device-timed step
            h = hk.hk_setup_nested(m.xyz, m.elems, m.is_boundary, p.coeff, p.k, p.elem_to_sub, p.n_sub, e2f_host,
                                   fine ** m.dim, p.overlap, args.fine_overlap, p.tau, prec, hk.HK_AS, p.restart,
                                   p.max_iters, sptr)
        else:
            h = hk.hk_setup(m.xyz, m.elems, m.is_boundary, p.coeff, p.k, p.elem_to_sub, p.n_sub, p.overlap, p.tau,
                            prec, hk.HK_TWO_LEVEL, hk.HK_AS, p.restart, p.max_iters, sptr)
        hk.hk_solve(h, rhs_host, p.tol)
        hk.hk_destroy(h)
        torch.cuda.synchronize()
        e2e_ms.append(1e3 * (time.perf_counter() - t0))
    e2e_t = max_over_ranks(sum(e2e_ms) / 1e3, world)
    e2e_value = len(e2e_ms) * s * world / e2e_t

    # ---- solve-only (operator resident, as in serving): both precision forms
    def solve_only(precision, n):
        h = setup_dev(precision)
        for _ in range(2):
            hk.hk_solve_device(h, d_rhs, d_u, p.tol)
        lat, its = [], None
        for _ in range(n):
            flush.fill_(1.0)
            a, b = ev(), ev()
            a.record(stream)
            r = hk.hk_solve_device(h, d_rhs, d_u, p.tol)
            b.record(stream)
            b.synchronize()
            lat.append(a.elapsed_time(b))
            its = int(r.iters[0])
        info = hk.hk_info(h)
        hk.hk_destroy(h)
        lat = np.array(lat)
        return {"solves_per_s": float(s * 1e3 / lat.mean()), "p50_ms": float(np.percentile(lat, 50)),
                "p99_ms": float(np.percentile(lat, 99)), "iterations": its, "setup_ms": info["setup_ms"][5]}

    so32 = solve_only(hk.HK_FP32_PRECOND, args.solve_reps)
    so64 = solve_only(hk.HK_FP64, args.solve_reps)
    sosp = solve_only(hk.HK_SPLIT_BF16_PRECOND, args.solve_reps)

    # ---- tensor-core local sweeps of the split-BF16 form against the FP32 CUDA-core sweeps, on one
    # apply of 16 right-hand sides (the multi-right-hand-side case the tensor cores are for)
    def sweeps_compare(n_rhs=16, reps=10):
        h = setup_dev(hk.HK_SPLIT_BF16_PRECOND)
        info = hk.hk_info(h)
        if info["tc_record_bytes"] == 0:
            hk.hk_destroy(h)
            return {"unavailable": "tensor-core sweeps not built for these subdomains"}
        v = np.random.default_rng(1).standard_normal((n_rhs, info["n_dofs"]))
        out = {"rhs_per_apply": n_rhs}
        for name, path in (("tensor_core", hk.HK_SWEEPS_TENSOR_CORE), ("cuda_core_fp32", hk.HK_SWEEPS_CUDA_CORE)):
            hk.hk_set_sweep_path(h, path)
            hk.hk_apply_precond(h, v)
            hk.hk_set_timing(h, True)
            for _ in range(reps):
                hk.hk_apply_precond(h, v)
            t = hk.hk_kernel_times(h)
            hk.hk_set_timing(h, False)
            out[name] = {k: 1e3 * t[k][0] / reps for k in ("local_apply", "coarse_solve", "scatter")}
        hk.hk_destroy(h)
        # MMA work per launch: every record entry (BF16 pair) meets 16 right-hand sides in three products
        flops = 3 * 2 * TC_NRHS * info["tc_record_bytes"] / 4
        tc_s = out["tensor_core"]["local_apply"] * 1e-6
        out["speedup_local_sweeps"] = out["cuda_core_fp32"]["local_apply"] / out["tensor_core"]["local_apply"]
        out["roofline"] = {"bound": "tensor", "kernel": "k_local_apply_tc", "achieved": flops / tc_s / 1e12,
                           "traffic": measured_traffic("k_local_apply_tc", f"{args.workload}_split_16rhs"),
                           "peak": BF16_PEAK, "unit": "TFLOP/s", "frac": flops / tc_s / 1e12 / BF16_PEAK,
                           "mma_tflop_per_launch": flops / 1e12, "record_bytes_per_launch": info["tc_record_bytes"],
                           "record_gbs": info["tc_record_bytes"] / tc_s / 1e9,
                           "peak_source": "MEASURED_PEAKS.json bf16_tflops (burst)",
                           "note": "a chain of about L/2 dependent level steps per subdomain, each a few dozen "
                                   "N = 16 MMAs: issue- and latency-bound, not throughput-bound"}
        return out

    tc_cmp = sweeps_compare()

    # ---- roofline from the live kernel timings of the timed steps
    info0, _, its0 = rec[0]
    kt0 = rec_t[0][1]
    pf = 8 if prec == hk.HK_FP64 else 4
    n, n0 = info0["n_dofs"], info0["n0"]
    It, ze = info0["dof_total"], info0["coarse_elems"]
    # algorithmic bytes of one apply of s right-hand sides: the banded-LU fill |I_i| (3 w_i + 1) of
    # every local factor (the least a local solve must stream), v read and z written in FP64, the
    # index and pull maps, Z_i for restriction and prolongation, E^{-1}
    nI_list, w_list = hk_sub_sizes(p, widths=True)
    fill = sum(nI * (3 * w + 1) for nI, w in zip(nI_list, w_list))
    bytes_local = fill * pf + s * n * 8 + It * 4
    bytes_coarse = 2 * ze * pf + n0 * n0 * pf
    bytes_scatter = s * n * 8 + It * 4
    agg = {k: [ms, c] for k, (ms, c) in kt0.items()}
    eig_ms, eig_gf, setup_ms = [], [], []
    for info, _, _ in rec:
        eig_ms.append(info["eigen_kernel_ms"][:3])
        eig_gf.append(info["eigen_kernel_gflop"][:3])
        setup_ms.append(info["setup_ms"][5])
    eig_mean = [statistics.mean(x[i] for x in eig_ms) for i in range(3)]
    eig_gflop = [statistics.mean(x[i] for x in eig_gf) for i in range(3)]
    hbm, src = peaks()
    per = {k: (v[0] / max(v[1], 1)) for k, v in agg.items()}
    # the coarse branch runs beside the local sweeps (forked stream): the apply takes the longer
    # of the two, then the scatter
    apply_ms = max(per["local_apply"], per.get("coarse_solve", 0.0)) + per["scatter"]
    apply_bytes = bytes_local + bytes_coarse + bytes_scatter
    roof_apply = {"bound": "hbm", "achieved": apply_bytes / (apply_ms * 1e-3) / 1e9, "peak": hbm, "unit": "GB/s",
                  "frac": apply_bytes / (apply_ms * 1e-3) / 1e9 / hbm,
                  "traffic": measured_traffic("k_local_apply", f"{args.workload}_{args.precision}"),
                  "traffic_kernel": "k_local_apply (the sweeps; the coarse branch and scatter are not included)",
                  "kernels": "k_local_apply || (k_restrict -> k_coarse_solve -> k_prolong), then k_scatter",
                  "bytes_per_apply": apply_bytes, "rhs_per_apply": s, "ms_per_apply": apply_ms,
                  "peak_source": src}
    # dominant kernel over the step: the eigen kernels of the setup vs the solve kernels
    tot = {k: v[0] for k, v in agg.items()}
    tot["eigen_inertia"], tot["eigen_lanczos"], tot["eigen_refine"] = eig_mean
    dom = max(tot, key=tot.get)
    if dom.startswith("eigen_"):
        # CUDA-core peaks from unit counts and the maximum SM clock (no measured figure exists for them):
        # FP32 152 SMs x 128 lanes x 2 flops x 2.07 GHz; FP64 152 SMs x 2 FMA per clock x 2 flops x 2.07 GHz
        i = ["eigen_inertia", "eigen_lanczos", "eigen_refine"].index(dom)
        kname = ["k_inertia", "k_lanczos", "k_refine"][i]
        fp32 = kname == "k_lanczos"
        peak_tf = 152 * (128 if fp32 else 2) * 2 * 2.07e9 / 1e12
        ach = eig_gflop[i] / tot[dom]  # GFLOP / ms = TFLOP/s
        roof = {"bound": "alu", "achieved": ach, "peak": peak_tf, "unit": "TFLOP/s", "frac": ach / peak_tf,
                "traffic": measured_traffic(kname, args.workload), "algorithmic_gflop": eig_gflop[i],
                "kernel": kname + (" (FP32 shift-invert block Lanczos)" if fp32 else " (FP64)"),
                "ms_per_launch": tot[dom],
                "peak_source": "derived: " + ("FP32 CUDA cores" if fp32 else "FP64 units") + " x 2.07 GHz",
                "note": {"k_inertia": "one CTA per subdomain; a chain of FP64 level steps",
                         "k_lanczos": "one CTA per subdomain; a latency-bound chain of level steps",
                         "k_refine": "one CTA per candidate cluster; FP64-pipe bound (block LU and sweeps of "
                                     "the shifted pencil) with a barrier chain per pivot"}[kname]}
    else:
        b = {"local_apply": bytes_local, "coarse_solve": bytes_coarse, "scatter": bytes_scatter}.get(dom)
        if b is None:
            b = bytes_local
        ach = b / (per[dom] * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": ach, "peak": hbm, "unit": "GB/s", "frac": ach / hbm, "traffic": None,
                "kernel": dom, "peak_source": src}
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": sum(step_ms) / len(step_ms), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded)",
            "config": workload_config(p, args.workload, args.precision, args.fine_parts, args.fine_overlap),
            "iterations": [int(x) for x in its0],
            "setup_phases_ms": dict(zip(["assembly", "decomposition", "local_factors", "eigen", "coarse"],
                                        [round(x, 3) for x in info0["setup_ms"][:5]])),
            "phases_ms": {"setup": statistics.mean(setup_ms),
                          "eigen_kernels": dict(zip(["inertia", "lanczos", "refine"], eig_mean)),
                          "eigen_kernels_gflop": dict(zip(["inertia", "lanczos", "refine"], eig_gflop)),
                          "solve": statistics.mean(step_ms) - statistics.mean(setup_ms)},
            "latency_ms": {"p50": float(np.percentile(step_ms, 50)), "p99": float(np.percentile(step_ms, 99))},
            "local_factors": {"twist_moved": info0["twist_moved"], "pivot_growth": info0["local_growth"][0],
                              "pivot_growth_middle_twist": info0["local_growth"][1],
                              "fine_subdomains": info0["fine_subdomains"]},
            "solve_only": {"fp32_precond": so32, "fp64": so64, "split_bf16": sosp},
            "split_bf16_local_sweeps": tc_cmp,
            "kernel_ms_per_launch": per, "roofline": roof, "roofline_apply": roof_apply,
            "e2e": {"value": e2e_value, "unit": "solves/s", "h2d_bytes_per_step": int(h2d),
                    "d2h_bytes_per_step": int(d2h)},
            "gpu_launches": int(launches), "clocks": clocks, "wall_s": wall,
            "solve_path": "one CUDA graph per solve (device-side loops)" if info0["graph_solves"] > 0
                          else "host-driven loop"}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = cpu_baseline(
            p, nested=(W.box_partition(m, args.fine_parts), args.fine_overlap) if args.fine_parts else None)
    if rank == 0:
        print(json.dumps(line), flush=True)


# ------------------------------------------------------------------ serving workload
def run_serving(args, world, rank, local):
    """24 cached operators behind hk_server_*: the operator cache is warmed once (one request per
    operator, setups timed), then the same 2,000-request recipe is replayed (a) as one burst, which
    measures capacity, and (b) as Poisson streams at fractions of that capacity, which measure latency.
    Every solve goes through the public serving calls, host right-hand sides in, host solutions out."""
    import torch

    from paper_2406_06283_gb300 import hk

    torch.cuda.set_device(local)
    ops = W.config_c5()
    prec = PRECISIONS[args.precision]
    budget = int(args.budget_gb * (1 << 30))
    srv = hk.hk_server_create(budget, n_slots=args.slots, max_batch_rhs=16)
    ids = [hk.server_add_problem(srv, p, prec) for p in ops]
    launches0 = hk.hk_kernel_launches()

    def replay(stream, burst):
        tickets = [None] * len(stream)
        t0 = time.perf_counter()

        def submit():
            for q, (ta, o, idx) in enumerate(stream):
                if not burst:
                    d = ta - (time.perf_counter() - t0)
                    if d > 0:
                        time.sleep(d)
                tickets[q] = hk.hk_server_submit(srv, ids[o], ops[o].rhs[idx], 1e-8)
        th = threading.Thread(target=submit)
        th.start()
        lat, first, last, nrhs, its, bad, refused = [], None, None, 0, [], 0, 0
        for q, (ta, o, idx) in enumerate(stream):
            while tickets[q] is None:
                time.sleep(0.0005)
            r = hk.hk_server_poll(srv, tickets[q], ids[o], len(idx), wait_ms=-1, raise_on_failure=False)
            inf = r.info
            lat.append(inf["end_ms"] - inf["submit_ms"])
            first = inf["submit_ms"] if first is None else min(first, inf["submit_ms"])
            last = inf["end_ms"] if last is None else max(last, inf["end_ms"])
            if r.status in (hk.HK_OK, hk.HK_NO_CONVERGENCE):
                nrhs += len(idx)  # solves answered; refused requests count in `refused`, not as solves
                its.extend(int(x) for x in r.iters)
            else:
                refused += 1
            bad += int(r.status != hk.HK_OK)
        th.join()
        span = (last - first) / 1e3
        return {"requests": len(stream), "rhs": nrhs, "solves_per_s": nrhs / span, "requests_per_s": len(stream) / span,
                "refused_requests": refused,
                "p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_iters": float(np.mean(its)), "not_converged": bad, "span_s": span}

    # warm the operator cache: one single-rhs request per operator
    t0 = time.perf_counter()
    warm = replay([(0.0, i, [0]) for i in range(len(ops))], burst=True)
    warm_s = time.perf_counter() - t0
    st_warm = hk.hk_server_get_stats(srv)
    sampler = ClockSampler(local)
    sampler.start()
    burst = replay(W.serving_stream(len(ops), args.requests, 1.0, seed=5), burst=True)
    rates = {}
    for frac in (0.5, 0.8):
        lam = frac * burst["requests_per_s"]
        rates[f"{frac:.1f}x_capacity"] = replay(W.serving_stream(len(ops), args.requests, lam, seed=5), burst=False)
        rates[f"{frac:.1f}x_capacity"]["arrival_rate_per_s"] = lam
    clocks = sampler.stop()
    launches = hk.hk_kernel_launches() - launches0
    stats = hk.hk_server_get_stats(srv)
    hk.hk_server_destroy(srv)
    n_avg = float(np.mean([p.mesh.n_dofs for p in ops]))
    line = {"metric": METRIC, "value": burst["solves_per_s"], "unit": "solves/s", "n_gpus": world,
            "steps": args.requests, "warmup": len(ops), "ms_per_step": 1e3 * burst["span_s"] / args.requests,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded)",
            "config": {"workload": "c5 serving: 24 cached operators (16 2D h in 1/128..1/512, k in [20,100], "
                                   "checkerboard a in 10^U[0,2]; 8 3D h=1/32 Kuhn tets, k=20, 4x4x4 boxes); "
                                   f"{args.requests} requests, 1-4 rhs each, tol 1e-8",
                       "slots": args.slots, "max_batch_rhs": 16, "budget_gb": args.budget_gb,
                       "precision_form": args.precision, "parallelism": "replicas",
                       "l2": "inputs of the stream exceed L2 (24 operators, several GB resident)"},
            "latency_ms": {"p50": burst["p50_ms"], "p99": burst["p99_ms"]},
            "serving": {"burst": burst, "poisson": rates, "warm_cache": {"seconds": warm_s, **warm},
                        "stats": stats, "setups_during_warm": st_warm["setups"]},
            "e2e": {"value": burst["solves_per_s"], "unit": "solves/s",
                    "h2d_bytes_per_step": int(8 * n_avg * 2.5), "d2h_bytes_per_step": int(8 * n_avg * 2.5),
                    "note": "value is already end to end: host rhs in, host u out, through hk_server_*"},
            "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = serving_cpu_baseline(ops)
    if rank == 0:
        print(json.dumps(line), flush=True)


def serving_cpu_baseline(ops, budget_s=25.0):
    """The oracle on the smallest operators of the serving set, setup + one solve each, until budget_s."""
    from oracle import solver as OS
    order = sorted(range(len(ops)), key=lambda i: ops[i].mesh.n_dofs * max(1, ops[i].mesh.dim - 1) ** 3)
    t0, done, names = time.perf_counter(), 0, []
    for i in order:
        p = ops[i]
        h = OS.setup_problem(p)
        OS.solve(h, p.rhs[:1], p.tol)
        done += 1
        names.append(p.name)
        if time.perf_counter() - t0 > budget_s:
            break
    el = time.perf_counter() - t0
    return {"value": done / el, "unit": "solves/s", "cores": os.cpu_count(), "kind": "oracle",
            "sample": f"setup + one solve of {done} serving operators ({', '.join(names)}), no cache reuse; "
                      f"numpy/scipy, BLAS threads up to {os.cpu_count()}"}


# ------------------------------------------------------------------ batched workload
def run_batched(args, world, rank, local):
    """64 independent instances (each: setup + solve of 1-8 right-hand sides) submitted at once through
    the serving calls to a fresh server: the worker slots overlap the instances on the device, each
    solve runs as one CUDA graph, and the apply's right-hand-side grouping is autotuned per instance.
    A step is the whole batch; every step builds a fresh server, so every setup is paid."""
    import torch

    from paper_2406_06283_gb300 import hk

    torch.cuda.set_device(local)
    probs = W.config_c4()
    prec = PRECISIONS[args.precision]
    budget = int(args.budget_gb * (1 << 30))
    nrhs = sum(p.rhs.shape[0] for p in probs)

    def batch(ps):
        srv = hk.hk_server_create(budget, n_slots=args.slots, max_batch_rhs=8)
        t0 = time.perf_counter()
        ids = [hk.server_add_problem(srv, p, prec) for p in ps]
        tickets = [hk.hk_server_submit(srv, i, p.rhs, p.tol) for i, p in zip(ids, ps)]
        res = [hk.hk_server_poll(srv, t, i, p.rhs.shape[0], raise_on_failure=False)
               for t, i, p in zip(tickets, ids, ps)]
        el = time.perf_counter() - t0
        st = hk.hk_server_get_stats(srv)
        hk.hk_server_destroy(srv)
        return el, res, st

    small = sorted(probs, key=lambda p: p.mesh.n_dofs)[:3]
    for _ in range(max(1, args.warmup)):
        batch(small)
    launches0 = hk.hk_kernel_launches()
    sampler = ClockSampler(local)
    sampler.start()
    times, last = [], None
    for _ in range(max(1, args.steps)):
        el, res, st = batch(probs)
        times.append(el)
        last = (res, st)
    clocks = sampler.stop()
    launches = hk.hk_kernel_launches() - launches0
    res, st = last
    t = max_over_ranks(sum(times), world)
    # solves answered per second (instances the library refuses are listed in the line, not counted)
    res0 = last[0]
    answered = sum(p.rhs.shape[0] for r, p in zip(res0, probs) if r.status in (hk.HK_OK, hk.HK_NO_CONVERGENCE))
    value = len(times) * answered * world / t
    lat = [r.info["end_ms"] - r.info["submit_ms"] for r in res]
    conv = sum(int((r.iters > 0).all() and r.status == hk.HK_OK) for r in res)
    # instances the library refuses or fails on are counted, not left out of the workload
    refused = [p.name for r, p in zip(res, probs) if r.status not in (hk.HK_OK, hk.HK_NO_CONVERGENCE)]
    solved_rhs = sum(p.rhs.shape[0] for r, p in zip(res, probs) if r.status in (hk.HK_OK, hk.HK_NO_CONVERGENCE))
    line = {"metric": METRIC, "value": value, "unit": "solves/s", "n_gpus": world, "steps": len(times),
            "warmup": max(1, args.warmup), "ms_per_step": 1e3 * sum(times) / len(times), "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None,
            "dtype": DTYPES[args.precision],
            "data": "synthetic (seeded)",
            "config": {"workload": f"c4 batched: {len(probs)} independent 2D instances (h in 1/128..1/384, "
                                   f"k in [20,80], checkerboard a in 10^U[0,2], 4..12 boxes per side), "
                                   f"{nrhs} right-hand sides, each instance set up and solved to 1e-8",
                       "slots": args.slots, "precision_form": args.precision, "parallelism": "replicas",
                       "l2": "64 instances, several GB resident: inputs exceed L2"},
            "latency_ms": {"p50": float(np.percentile(lat, 50)), "p99": float(np.percentile(lat, 99))},
            "batched": {"instances": len(probs), "rhs": nrhs, "converged_instances": conv,
                        "refused_or_failed": refused, "rhs_of_answered_instances": solved_rhs,
                        "mean_iters": float(np.mean([x for r in res for x in r.iters])),
                        "setups": st["setups"], "batches": st["batches"], "bytes_peak": st["bytes_peak"]},
            "e2e": {"value": value, "unit": "solves/s",
                    "h2d_bytes_per_step": int(sum(p.rhs.nbytes + p.mesh.xyz.nbytes + p.mesh.elems.nbytes // 2 +
                                                  p.coeff.nbytes for p in probs)),
                    "d2h_bytes_per_step": int(sum(p.rhs.nbytes for p in probs)),
                    "note": "value is already end to end: host inputs in, host solutions out, through hk_server_*"},
            "gpu_launches": int(launches), "clocks": clocks}
    if rank == 0 and world == 1 and not args.no_cpu_baseline:
        line["cpu_baseline"] = serving_cpu_baseline(probs)
    if rank == 0:
        print(json.dumps(line), flush=True)


def hk_sub_sizes(p, widths=False):
    """|dof(Omega_i)| of every subdomain (and, with widths, the widest level set of each, the band
    width w_i of B_i in level order), read back through the C ABI."""
    from paper_2406_06283_gb300 import hk
    h = hk.setup_problem(p, precision=hk.HK_FP32_PRECOND)
    subs = [hk.hk_get_subdomain(h, i) for i in range(p.n_sub)]
    hk.hk_destroy(h)
    out = [sd["dof"].size for sd in subs]
    if widths:
        return out, [int(np.diff(sd["level_ptr"]).max()) for sd in subs]
    return out


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=10)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="c2", choices=["c1", "c2", "c3", "c4", "c5"])
    ap.add_argument("--requests", type=int, default=2000, help="c5: requests per replay")
    ap.add_argument("--slots", type=int, default=4, help="c5: server worker slots")
    ap.add_argument("--budget-gb", type=float, default=64.0, help="c5: server device-memory budget")
    ap.add_argument("--precision", default="fp32", choices=["fp32", "fp64", "split"])
    ap.add_argument("--solve-reps", type=int, default=20)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--fine-parts", type=int, default=0,
                    help="nested decompositions (Sec. 2.3): fine boxes per axis inside the coarse subdomains (0: one "
                         "decomposition)")
    ap.add_argument("--fine-overlap", type=int, default=2, help="overlap layers of the fine subdomains")
    ap.add_argument("--profile-sweeps", action="store_true",
                    help="only 16-right-hand-side applies, tensor-core then CUDA-core sweeps, twice each (split form; "
                         "for ncu captures of the sweep kernels)")
    ap.add_argument("--profile-run", action="store_true",
                    help="one warm-up step and one step with the solve's kernels launched one by one, "
                         "nothing else (for ncu captures)")
    args = ap.parse_args()
    world, rank, local = dist_init()
    if args.impl == "reference":
        run_reference(args, world, rank)
    elif args.workload == "c5":
        run_serving(args, world, rank, local)
    elif args.workload == "c4":
        run_batched(args, world, rank, local)
    else:
        run_ours(args, world, rank, local)
    if world > 1:
        import torch.distributed as dist
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
