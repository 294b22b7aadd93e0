"""Serving loop: admission by memory budget, continuous batching, overlap of
batches on several workers (CPU, with a fake batch executor), and -- on the
GPU -- every result the same alone and in the mix."""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
from paper_1610_09411_gb300.serve import CensusServer, footprint_bytes, poisson_arrivals, replay


def _fake_run(log, delay=0.02):
    active = {"now": 0, "peak": 0}
    lk = threading.Lock()

    def run(batch, stream):
        with lk:
            active["now"] += 1
            active["peak"] = max(active["peak"], active["now"])
        log.append([r.n for r in batch])
        time.sleep(delay)
        with lk:
            active["now"] -= 1
        return [{"n": r.n, "m": int(r.row_ptr[-1]) // 2} for r in batch]
    return run, active


def test_all_requests_complete_with_their_own_result():
    log = []
    run, _ = _fake_run(log)
    srv = CensusServer(budget_bytes=1e12, workers=2, run_batch=run, upload=lambda r: None)
    graphs = [gg.erdos_renyi(20 + k, 0.2, k) for k in range(30)]
    futs = [srv.submit(g.row_ptr, g.col, g.n) for g in graphs]
    res = [f.result(timeout=10) for f in futs]
    srv.close()
    assert [r["n"] for r in res] == [g.n for g in graphs]
    assert [r["m"] for r in res] == [g.m for g in graphs]
    assert sum(len(b) for b in log) == 30


def test_requests_arriving_during_a_batch_join_a_later_batch_and_batches_overlap():
    log = []
    run, active = _fake_run(log, delay=0.05)
    srv = CensusServer(budget_bytes=1e12, workers=3, run_batch=run, upload=lambda r: None)
    graphs = [gg.erdos_renyi(10, 0.3, k) for k in range(40)]
    futs = replay(srv, graphs, poisson_arrivals(400.0, len(graphs), 1))
    for f in futs:
        f.result(timeout=10)
    srv.close()
    assert len(log) > 1                        # more than one batch formed
    assert max(len(b) for b in log) > 1        # later arrivals were batched together
    assert active["peak"] > 1                  # batches overlapped


def test_admission_respects_the_memory_budget():
    g = gg.erdos_renyi(50, 0.2, 3)
    need = footprint_bytes(g.n, g.m)
    inflight = {"max": 0}
    log = []
    run, _ = _fake_run(log, delay=0.02)
    srv = CensusServer(budget_bytes=2.5 * need, workers=4, run_batch=run, upload=lambda r: None)

    def watch():
        while not srv.closed:
            inflight["max"] = max(inflight["max"], srv.in_use)
            time.sleep(0.001)
    t = threading.Thread(target=watch)
    t.start()
    futs = [srv.submit(g.row_ptr, g.col, g.n) for _ in range(12)]
    for f in futs:
        f.result(timeout=10)
    srv.close()
    t.join()
    assert inflight["max"] <= 2.5 * need
    assert srv.in_use == 0


def test_oversized_request_is_rejected_not_hung():
    srv = CensusServer(budget_bytes=1000, workers=1, run_batch=lambda b, s: [None] * len(b), upload=lambda r: None)
    g = gg.complete(10)
    f = srv.submit(g.row_ptr, g.col, g.n)
    with pytest.raises(MemoryError):
        f.result(timeout=5)
    srv.close()


@pytest.mark.gpu
def test_gpu_results_alone_and_in_the_mix_are_identical():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1610_09411_gb300 import build
    build.build()
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.chung_lu(int(n), 2.3, 8, 200, s) for s, n in enumerate([200, 3000, 50, 800, 12000, 400, 90, 2500])]
    graphs += [gg.erdos_renyi(120, 0.1, 7), gg.complete(30), gg.empty(3)]
    alone = [esc.census(g.row_ptr, g.col, n=g.n) for g in graphs]
    srv = CensusServer(budget_bytes=120e9, workers=3)
    futs = replay(srv, graphs, poisson_arrivals(2000.0, len(graphs), 5))
    mixed = [f.result(timeout=120) for f in futs]
    srv.close()
    for a, b in zip(alone, mixed):
        for k in ("c3", "c4", "c5", "n3", "n4", "n5"):
            assert a[k] == b[k]
