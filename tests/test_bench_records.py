"""Host logic of bench.py's roofline `traffic` field (no GPU): the DRAM bytes of a kernel come from the ncu
record in profiles/dram_traffic.txt, and only while the CUDA file that defines the kernel is the one the
counters were taken from (the record carries that file's sha256).  A record of a changed file, of an
unknown kernel or of another workload gives null."""
import os
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

import bench  # noqa: E402


def _records():
    out = []
    for ln in open(bench.TRAFFIC_PATH).read().splitlines():
        f = ln.split()
        if f and not ln.startswith("#"):
            out.append(f)
    return out


def test_every_record_names_a_defined_kernel():
    recs = _records()
    assert recs
    for f in recs:
        assert len(f) == 4, f
        kernel, workload, digest, nbytes = f
        path = bench.kernel_source(kernel)
        assert path is not None, kernel
        assert "__global__" in open(path).read()
        assert len(digest) == 16 and int(nbytes) > 0


def test_the_defining_file_not_a_file_that_only_names_the_kernel():
    # hk_eigen.cu names k_lanczos and k_inertia in its comments; they are defined in hk_lanczos.cu
    assert bench.kernel_source("k_lanczos").endswith("hk_lanczos.cu")
    assert bench.kernel_source("k_inertia").endswith("hk_lanczos.cu")
    assert bench.kernel_source("k_refine").endswith("hk_eigen.cu")
    assert bench.kernel_source("k_local_apply").endswith("hk_local.cu")
    assert bench.kernel_source("k_local_apply_tc").endswith("hk_tc.cu")
    assert bench.kernel_source("k_no_such_kernel") is None


def test_record_used_only_while_the_source_is_unchanged(tmp_path, monkeypatch):
    dig = bench.source_digest("k_refine")
    stale = "0" * 16 if dig != "0" * 16 else "1" * 16
    p = tmp_path / "dram_traffic.txt"
    p.write_text(f"# header\nk_refine c2 {dig} 1234\nk_lanczos c2 {stale} 5678\n")
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(p))
    assert bench.measured_traffic("k_refine", "c2") == 1234
    assert bench.measured_traffic("k_refine", "c3") is None       # another workload
    assert bench.measured_traffic("k_lanczos", "c2") is None      # file changed since the counters
    assert bench.measured_traffic("k_inertia", "c2") is None      # no record
    monkeypatch.setattr(bench, "TRAFFIC_PATH", str(tmp_path / "missing.txt"))
    assert bench.measured_traffic("k_refine", "c2") is None
