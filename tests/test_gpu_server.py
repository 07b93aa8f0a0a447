"""The serving calls (hk_server_*): cached operators, admission by device memory, continuous batching.

Each served result is compared with hk_solve of the same right-hand side on a handle of its own, alone.
The solve treats every right-hand side independently with the same arithmetic whatever the batch
(per-right-hand-side reductions, state and stopping), so the comparison is exact: equal iteration
counts and bitwise-equal solutions.  The parity of hk_solve itself with the oracle is covered by
test_gpu_parity.py; here the served FP64 results are also checked against the oracle's solution.
"""
import threading
import time

import numpy as np
import pytest

from oracle import solver as OS
from paper_2406_06283_gb300 import hk
from paper_2406_06283_gb300 import workloads as W

pytestmark = pytest.mark.gpu


def _ops():
    return [W.small_problem(cells=24, parts=3, k=12.0, overlap=2, checker=3, seed=8),
            W.small_problem(cells=32, parts=4, k=15.0, overlap=2, checker=4, seed=12),
            W.small_problem_3d(cells=8, parts=2, k=4.0, overlap=1)]


def _requests(ops, n, seed):
    rng = np.random.default_rng(seed)
    out = []
    for q in range(n):
        o = int(rng.integers(len(ops)))
        s = int(rng.integers(1, 5))
        rhs = np.stack([W.normal(W.stream_seed(500 + seed, q, r), ops[o].mesh.n_dofs) for r in range(s)])
        out.append((o, rhs))
    return out


def _alone(ops, reqs, precision):
    hs = [hk.setup_problem(p, precision=precision) for p in ops]
    res = [hk.hk_solve(hs[o], rhs, 1e-8) for o, rhs in reqs]
    for h in hs:
        hk.hk_destroy(h)
    return res


@pytest.mark.parametrize("precision", [hk.HK_FP64, hk.HK_FP32_PRECOND])
def test_served_results_equal_alone_results(precision):
    ops = _ops()
    reqs = _requests(ops, 14, seed=1)
    want = _alone(ops, reqs, precision)
    srv = hk.hk_server_create(8 << 30, n_slots=3, max_batch_rhs=8)
    ids = [hk.server_add_problem(srv, p, precision) for p in ops]
    # submit from a second thread with small gaps while the first requests already run
    tickets = [None] * len(reqs)

    def submit():
        for q, (o, rhs) in enumerate(reqs):
            tickets[q] = hk.hk_server_submit(srv, ids[o], rhs, 1e-8)
            time.sleep(0.002)
    th = threading.Thread(target=submit)
    th.start()
    th.join()
    batched = 0
    for q, (o, rhs) in enumerate(reqs):
        got = hk.hk_server_poll(srv, tickets[q], ids[o], rhs.shape[0], wait_ms=-1)
        assert got.status == hk.HK_OK
        np.testing.assert_array_equal(got.iters, want[q].iters)
        np.testing.assert_array_equal(got.u, want[q].u)
        np.testing.assert_array_equal(got.true_rel_res, want[q].true_rel_res)
        assert got.info["end_ms"] >= got.info["start_ms"] >= got.info["submit_ms"]
        batched += got.info["batch_rhs"] > rhs.shape[0]
    st = hk.hk_server_get_stats(srv)
    assert st["completed"] == len(reqs) and st["failed"] == 0
    assert st["setups"] == len(ops)            # one setup per operator, the rest served from the cache
    assert st["cache_hits"] == st["batches"] - len(ops)
    assert st["bytes_peak"] <= st["budget"]
    hk.hk_server_destroy(srv)
    if precision == hk.HK_FP64:  # and the served solutions are the oracle's
        o0 = OS.setup_problem(ops[0])
        for q, (o, rhs) in enumerate(reqs):
            if o == 0:
                for r in range(rhs.shape[0]):
                    x = OS.solve(o0, rhs[r:r + 1], 1e-8)[0].x
                    assert np.linalg.norm(want[q].u[r] - x) <= 1e-7 * np.linalg.norm(x)


def test_identical_operator_is_cached_once():
    p = _ops()[0]
    srv = hk.hk_server_create(4 << 30, n_slots=2)
    a = hk.server_add_problem(srv, p)
    b = hk.server_add_problem(srv, p)
    assert a == b
    t1 = hk.hk_server_submit(srv, a, p.rhs)
    r1 = hk.hk_server_poll(srv, t1, a, 1)
    t2 = hk.hk_server_submit(srv, a, p.rhs)
    r2 = hk.hk_server_poll(srv, t2, a, 1)
    assert r1.info["setup_ran"] == 1 and r2.info["setup_ran"] == 0
    np.testing.assert_array_equal(r1.u, r2.u)
    with pytest.raises(hk.HKError) as e:
        hk.hk_server_poll(srv, t2, a, 1)
    assert e.value.status == hk.HK_BAD_ARG      # a ticket is forgotten once its result is read
    hk.hk_server_destroy(srv)


def test_budget_evicts_idle_operators_and_rejects_what_never_fits():
    ops = _ops()[:2]
    n1 = max(p.mesh.n_dofs for p in ops)
    # room for the first setup of the larger operator (24 KiB per dof before it was ever measured,
    # plus one right-hand side's solve workspace) and 64 KiB more: not for the other operator resident too
    # (each request brings one right-hand side: capacity S = 1)
    ws = 8 * ((2 * 50 + 6) * n1 + 51 * 54 + 1000) + (1 << 20)
    budget = 24576 * n1 + ws + (64 << 10)
    srv = hk.hk_server_create(budget, n_slots=2)
    ids = [hk.server_add_problem(srv, p) for p in ops]
    order = [0, 1, 0]
    res = []
    for o in order:
        t = hk.hk_server_submit(srv, ids[o], ops[o].rhs)
        res.append(hk.hk_server_poll(srv, t, ids[o], 1))
    st = hk.hk_server_get_stats(srv)
    assert st["evictions"] >= 1 and st["setups"] == 3 and st["bytes_peak"] <= budget
    for o, r in zip(order, res):
        assert r.status == hk.HK_OK and r.true_rel_res[0] <= 1e-8
    np.testing.assert_array_equal(res[0].u, res[2].u)   # rebuilt operator, same result
    hk.hk_server_destroy(srv)
    tiny = hk.hk_server_create(1 << 20, n_slots=1)
    a = hk.server_add_problem(tiny, ops[0])
    t = hk.hk_server_submit(tiny, a, ops[0].rhs)
    with pytest.raises(hk.HKError) as e:
        hk.hk_server_poll(tiny, t, a, 1)
    assert e.value.status == hk.HK_OOM
    hk.hk_server_destroy(tiny)
