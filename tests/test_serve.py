"""Serving loop: admission by memory budget, continuous batching, overlap of
batches on several workers (CPU, with a fake batch executor), and -- on the
GPU -- every result the same alone and in the mix."""
import threading
import time

import numpy as np
import pytest

import graphgen as gg
from paper_1610_09411_gb300.serve import CensusServer, footprint_bytes, poisson_arrivals, replay, triangle_bound


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


def test_triangle_bound_holds_and_lists_are_charged():
    """The degree-only bound is at least the true triangle count (oracle), so
    the footprint charges at least the 36 B per triangle the lists take."""
    import oracle
    for g in (gg.complete(40), gg.erdos_renyi(200, 0.3, 2), gg.chung_lu(2000, 2.1, 12, 300, 4),
              gg.complete_bipartite(20, 30), gg.disjoint_union([gg.complete(25), gg.star(60)])):
        T = oracle.census(g)["n3"][3]
        tb = triangle_bound(g.row_ptr, g.col)
        assert tb >= T
        deg = np.diff(g.row_ptr)
        assert footprint_bytes(g.n, g.m, tb, int(deg.max())) >= 36 * T
    assert triangle_bound(gg.complete(40).row_ptr, gg.complete(40).col) == 40 * 39 * 38 // 6


def test_admission_with_triangle_dense_requests_stays_in_budget():
    """Complete graphs (every edge in n - 2 triangles): in_use never exceeds
    the budget while requests overlap."""
    graphs = [gg.complete(k) for k in (60, 80, 100, 70, 90, 100, 60, 80)]
    needs = []
    for g in graphs:
        tb = triangle_bound(g.row_ptr, g.col)
        assert tb == g.n * (g.n - 1) * (g.n - 2) // 6
        needs.append(footprint_bytes(g.n, g.m, tb, g.n - 1))
    budget = 2.2 * max(needs)
    peak = {"max": 0}
    run, _ = _fake_run([], delay=0.02)
    srv = CensusServer(budget_bytes=budget, workers=4, run_batch=run, upload=lambda r: None)

    def watch():
        while not srv.closed:
            peak["max"] = max(peak["max"], srv.in_use)
            time.sleep(0.0005)
    t = threading.Thread(target=watch)
    t.start()
    futs = [srv.submit(g.row_ptr, g.col, g.n) for g in graphs]
    for f in futs:
        f.result(timeout=10)
    srv.close()
    t.join()
    assert 0 < peak["max"] <= budget
    assert srv.in_use == 0


def test_malformed_row_pointer_rejected_on_submit():
    srv = CensusServer(budget_bytes=1e12, workers=1, run_batch=lambda b, s: [None] * len(b), upload=lambda r: None)
    col = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)
    for rp in ([0, 4, 2, 6], [0, 2, 4, 9], [1, 2, 4, 6]):
        with pytest.raises(ValueError):
            srv.submit(np.array(rp, dtype=np.int64), col, 3).result(timeout=5)
    srv.close()


def test_admission_respects_the_memory_budget():
    g = gg.erdos_renyi(50, 0.2, 3)
    need = footprint_bytes(g.n, g.m, triangle_bound(g.row_ptr, g.col), int(np.diff(g.row_ptr).max()))
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
def test_gpu_results_alone_and_in_the_mix_equal_the_oracle():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1610_09411_gb300 import build
    build.build()
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.chung_lu(int(n), 2.3, 8, 200, s) for s, n in enumerate([200, 3000, 50, 800, 12000, 400, 90, 2500])]
    graphs += [gg.erdos_renyi(120, 0.1, 7), gg.complete(30), gg.empty(3)]
    import oracle
    want = [oracle.census(g) for g in graphs]
    alone = [esc.census(g.row_ptr, g.col, n=g.n) for g in graphs]
    srv = CensusServer(budget_bytes=120e9, workers=3)
    futs = replay(srv, graphs, poisson_arrivals(2000.0, len(graphs), 5))
    mixed = [f.result(timeout=120) for f in futs]
    srv.close()
    for w, a, b in zip(want, alone, mixed):
        for k in ("c3", "c4", "c5", "n3", "n4", "n5"):
            assert b[k] == w[k]          # served result = the oracle's
            assert a[k] == w[k]          # the census alone = the oracle's


@pytest.mark.gpu
def test_concurrent_censuses_with_heavy_pair_items_equal_the_oracle():
    """Censuses on three host threads at once, each on its own stream, over
    graphs whose heavy pair items use shared-memory windows of different
    widths (the launch limits one thread sets must hold for the others'
    launches); every result equals the oracle's."""
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    from paper_1610_09411_gb300 import build
    build.build()
    from paper_1610_09411_gb300 import escape as esc
    import oracle
    graphs = [gg.chung_lu(20000, 2.1, 10, 2000, 8), gg.chung_lu(6000, 2.1, 12, 1500, 3), gg.config_rmat(13, 2),
              gg.chung_lu(2500, 2.1, 14, 1200, 5)]
    want = [oracle.census(g) for g in graphs]
    errors, done = [], []

    def worker(t):
        try:
            torch.cuda.set_device(0)
            st = torch.cuda.Stream()
            for rep in range(3):
                for k in range(len(graphs)):
                    idx = (k + t + rep) % len(graphs)
                    g = graphs[idx]
                    got = esc.census(g.row_ptr, g.col, n=g.n, stream=st.cuda_stream)
                    for key in ("c3", "c4", "c5", "n3", "n4", "n5"):
                        assert got[key] == want[idx][key], (t, rep, idx, key)
                    done.append(idx)
        except Exception as e:            # reported by the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(t,)) for t in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join(timeout=600)
    assert not errors, errors[0]
    assert len(done) == 3 * 3 * len(graphs)
