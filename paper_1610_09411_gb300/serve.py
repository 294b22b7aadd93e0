"""Census serving with continuous batching on one GPU.

Requests (graphs as host CSR arrays) arrive at any time.  A request is
admitted when its estimated device footprint fits in what is left of the
device-memory budget; on admission its CSR is copied to the device and stays
resident until its result is out.  Worker threads, each with its own CUDA
stream, repeatedly take every admitted request that is not yet running (up to
a batch cap) and count them in one fused call of the batched census
(escape_census5_batch), so several batches run on the device at once and a
request that arrives while others are being counted joins the next batch.
Each result is the same as the graph's census alone: the batched pass keeps a
separate exact accumulator row per graph.

The execution step is injectable (``run_batch``) so the admission and
batching logic can be exercised without a GPU.
"""
from __future__ import annotations

import threading
import time
from collections import deque
from concurrent.futures import Future
from dataclasses import dataclass, field

import numpy as np


def footprint_bytes(n: int, m: int, sms: int = 152, cta_per_sm: int = 2) -> int:
    """Conservative device bytes for the census of one graph (n vertices, m
    edges): the CSR and its renamed copy, per-edge arrays and common-neighbour
    lists (bounded by the edge count times a triangle factor), and the sweep
    scratch that grows with n: per persistent CTA, 4 B per vertex for each of
    the tagged 4-cycle, pair and 5-cycle counters (the pair sweep runs three
    CTAs per SM), 8 B for the 5-cycle P2 counters and their list, and 8 B for
    the wheel counters of large centres (their degree is at most n).  Used for
    admission only."""
    nnz = 2 * m
    per_edge = nnz * (4 + 4 + 8 + 8 + 8 + 8 + 8 + 8)      # col x2, rev, T, K4, C4, offsets x2
    lists = nnz * 4 * 12                                    # id and position lists (triangle factor)
    per_vertex = n * 8 * 12
    sweep = n * sms * ((4 + 4 + 8) * cta_per_sm + 4 * 3 + 8 * 2)
    return int(per_edge + lists + per_vertex + sweep + (64 << 20))


@dataclass
class Request:
    n: int
    row_ptr: np.ndarray
    col: np.ndarray
    future: Future
    t_arrive: float
    bytes: int
    t_admit: float = 0.0
    t_start: float = 0.0
    t_finish: float = 0.0
    device: tuple = field(default=None, repr=False)   # resident device copies (row_ptr, col)


class CensusServer:
    def __init__(self, budget_bytes: float = 120e9, workers: int = 2, max_batch: int = 512,
                 max_batch_edges: int = 20_000_000, run_batch=None, upload=None, device=0):
        self.budget = int(budget_bytes)
        self.in_use = 0
        self.max_batch = max_batch
        self.max_batch_edges = max_batch_edges
        self.waiting: deque[Request] = deque()      # arrived, not admitted
        self.admitted: deque[Request] = deque()     # resident, not running
        self.lock = threading.Condition()
        self.closed = False
        self.device = device
        self._gpu = run_batch is None
        self._run_batch = run_batch or self._gpu_run_batch
        self._upload = upload or self._gpu_upload
        self.completed: list[Request] = []
        self.batches: list[int] = []
        self.workers = [threading.Thread(target=self._worker, args=(k,), daemon=True) for k in range(workers)]
        for t in self.workers:
            t.start()

    # ------------------------------------------------------------------ client side
    def submit(self, row_ptr, col, n: int | None = None) -> Future:
        row_ptr = np.ascontiguousarray(row_ptr, dtype=np.int64)
        col = np.ascontiguousarray(col, dtype=np.int32)
        n = len(row_ptr) - 1 if n is None else int(n)
        m = int(row_ptr[-1]) // 2 if n > 0 else 0
        fut: Future = Future()
        req = Request(n, row_ptr, col, fut, time.perf_counter(), footprint_bytes(n, m))
        if req.bytes > self.budget:
            fut.set_exception(MemoryError(f"request needs ~{req.bytes} B, budget is {self.budget} B"))
            return fut
        with self.lock:
            if self.closed:
                raise RuntimeError("server closed")
            self.waiting.append(req)
            self._admit_locked()
            self.lock.notify_all()
        return fut

    def close(self, wait: bool = True):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        if wait:
            for t in self.workers:
                t.join()

    # ------------------------------------------------------------------ internals
    def _admit_locked(self):
        # FIFO: the head waits until it fits, later requests do not overtake it
        while self.waiting and self.in_use + self.waiting[0].bytes <= self.budget:
            req = self.waiting.popleft()
            self.in_use += req.bytes
            req.t_admit = time.perf_counter()
            try:
                req.device = self._upload(req)
            except Exception as e:                       # upload failed: release and report
                self.in_use -= req.bytes
                req.future.set_exception(e)
                continue
            self.admitted.append(req)

    def _take_batch_locked(self):
        batch, edges = [], 0
        while self.admitted and len(batch) < self.max_batch:
            r = self.admitted[0]
            e = int(r.row_ptr[-1]) if r.n > 0 else 0
            if batch and edges + e > self.max_batch_edges:
                break
            batch.append(self.admitted.popleft())
            edges += e
        return batch

    def _worker(self, k: int):
        stream = self._make_stream()
        while True:
            with self.lock:
                while not self.admitted and not (self.closed and not self.waiting):
                    self.lock.wait(timeout=0.05)
                if not self.admitted and self.closed and not self.waiting:
                    return
                batch = self._take_batch_locked()
            if not batch:
                continue
            t0 = time.perf_counter()
            for r in batch:
                r.t_start = t0
            try:
                results = self._run_batch(batch, stream)
                err = None
            except Exception as e:   # the whole batch failed
                results, err = None, e
            t1 = time.perf_counter()
            with self.lock:
                for i, r in enumerate(batch):
                    r.t_finish = t1
                    r.device = None
                    self.in_use -= r.bytes
                    self.completed.append(r)
                self.batches.append(len(batch))
                self._admit_locked()
                self.lock.notify_all()
            for i, r in enumerate(batch):
                if err is not None:
                    r.future.set_exception(err)
                else:
                    r.future.set_result(results[i])

    def _make_stream(self):
        if not self._gpu:
            return None
        import torch
        torch.cuda.set_device(self.device)
        return torch.cuda.Stream()

    def _gpu_upload(self, req: Request):
        import torch
        with torch.cuda.device(self.device):
            rp = torch.from_numpy(req.row_ptr).to(f"cuda:{self.device}", non_blocking=False)
            col = torch.from_numpy(req.col if req.col.size else np.zeros(0, np.int32)).to(f"cuda:{self.device}")
        return rp, col

    def _gpu_run_batch(self, batch, stream):
        import torch
        from . import escape as esc
        with torch.cuda.device(self.device), torch.cuda.stream(stream):
            sizes = [r.n for r in batch]
            voff = np.zeros(len(batch) + 1, dtype=np.int64)
            voff[1:] = np.cumsum(sizes)
            parts, base = [], 0
            for r in batch:
                rp, _ = r.device
                parts.append(rp[:-1] + base)
                base += int(r.row_ptr[-1]) if r.n > 0 else 0
            dev = f"cuda:{self.device}"
            rp_all = torch.cat(parts + [torch.tensor([base], dtype=torch.int64, device=dev)])
            cols = [r.device[1] for r in batch]
            col_all = torch.cat(cols) if cols else torch.zeros(0, dtype=torch.int32, device=dev)
            dvoff = torch.from_numpy(voff).to(dev)
            stream.synchronize()
            return esc.escape_census5_batch(dvoff, rp_all, col_all, stream=stream.cuda_stream)

    # ------------------------------------------------------------------ reporting
    def latency_stats(self):
        lat = np.array([r.t_finish - r.t_arrive for r in self.completed]) * 1000.0
        if lat.size == 0:
            return {}
        return {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
                "mean_ms": float(lat.mean()), "count": int(lat.size),
                "mean_batch": float(np.mean(self.batches)) if self.batches else 0.0}


def poisson_arrivals(rate: float, count: int, seed: int) -> np.ndarray:
    """Arrival offsets (seconds) of a Poisson stream: exponential gaps from a
    seeded generator (request timing only, not graph content)."""
    rng = np.random.default_rng(seed)
    return np.cumsum(rng.exponential(1.0 / rate, size=count))


def replay(server: CensusServer, graphs, arrivals) -> list:
    """Submit graphs at the given arrival offsets (real time); returns futures."""
    t0 = time.perf_counter()
    futs = []
    for g, at in zip(graphs, arrivals):
        delay = t0 + at - time.perf_counter()
        if delay > 0:
            time.sleep(delay)
        futs.append(server.submit(g.row_ptr, g.col, g.n))
    return futs
