"""The multi-rank path of bench.py on the CPU: two gloo ranks (spawned processes, rendezvous on
127.0.0.1) run the helpers bench.py uses under torchrun -- rank discovery from the environment, the
barrier around the timed region and the maximum of the per-rank times -- and must agree on the job's
time.  The solver itself runs as one independent replica per rank (no collective on the data path),
so these helpers are the whole of the multi-rank logic."""
import multiprocessing as mp
import os
import socket
import sys

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket(socket.AF_INET, socket.SOCK_STREAM) as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, q):
    # CPU ranks even on a machine with GPUs: bench.py picks gloo when no device is visible
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world),
                      LOCAL_RANK=str(rank), CUDA_VISIBLE_DEVICES="")
    sys.path.insert(0, ROOT)
    try:
        import bench
        w, r, local = bench.dist_init()
        bench.barrier(w)
        t = bench.max_over_ranks(1.25 * (rank + 1), w)  # per-rank "times" 1.25 s and 2.5 s
        bench.barrier(w)
        import torch.distributed as dist
        backend = dist.get_backend()
        dist.destroy_process_group()
        q.put((rank, w, r, local, t, backend))
    except Exception as e:  # noqa: BLE001
        q.put((rank, "error", repr(e)))


def test_two_gloo_ranks_agree_on_the_job_time():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    out = {}
    for _ in range(2):
        item = q.get(timeout=120)
        out[item[0]] = item
    for p in procs:
        p.join(timeout=60)
    for rank in (0, 1):
        assert out[rank][1] != "error", out[rank]
        _, w, r, local, t, backend = out[rank]
        assert (w, r, local) == (2, rank, rank)
        assert t == 2.5  # both ranks see the slower rank's time
        assert backend == "gloo"
