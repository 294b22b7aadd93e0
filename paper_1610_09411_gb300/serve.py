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

Batches are also capped by predicted GPU time: every request carries the
census time the run-time model (predict.py, the paper's fit of run time to
basis counts, here from counts of the CSR) predicts for it, and a batch stops
growing at max_batch_seconds of predicted work.

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

from .predict import Predictor, host_counts


def triangle_bound(row_ptr: np.ndarray, col: np.ndarray) -> int:
    """Upper bound on the triangle count T from the degrees alone: an edge
    {u, v} lies in at most min(d_u, d_v) - 1 triangles and every triangle has
    three edges, so 3T <= sum over edges of (min(d_u, d_v) - 1)."""
    n = len(row_ptr) - 1
    if n <= 0 or len(col) == 0:
        return 0
    deg = np.diff(row_ptr).astype(np.int64)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    per_entry = np.minimum(deg[src], deg[col.astype(np.int64)]) - 1   # each edge appears twice
    return int(per_entry.clip(min=0).sum()) // 6


def footprint_bytes(n: int, m: int, tri_bound: int | None = None, max_deg: int | None = None,
                    sms: int = 152, cta_per_sm: int = 2) -> int:
    """Conservative device bytes for the census of one graph (n vertices, m
    edges, at most tri_bound triangles, largest degree max_deg): the CSR and
    its renamed copy and per-edge arrays; the common-neighbour lists, 3T ids
    and 6T positions (36 B per triangle); and the sweep scratch: per vertex, 8 B
    for each persistent CTA of the 4-cycle and 5-cycle sweeps (tagged counters)
    plus 8 B for the 5-cycle P2 counters and their list, 8 B per CTA slot of
    the pair sweep's counter arrays; per unit of the largest degree, the
    per-CTA wheel counters and common-neighbour hash tables.  Without a
    triangle bound, the lists are charged as if every edge were in max_deg
    triangles.  Used for admission only; the library's cache of released
    buffers (up to 8 GiB) and its fixed 8 MiB no-allocation array are not
    part of it."""
    nnz = 2 * m
    if max_deg is None:
        max_deg = n
    if tri_bound is None:
        tri_bound = m * max(max_deg - 1, 0) // 3
    grid = sms * cta_per_sm
    per_edge = nnz * (4 + 4 + 8 + 8 + 8 + 8 + 8 + 8)      # col x2, rev, T, K4, C4, offsets x2
    lists = 36 * tri_bound
    per_vertex = n * 8 * 12
    sweep = n * (grid * (8 + 8 + 8) + 8 * sms * 4) + max_deg * grid * (8 + 16)
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
    predicted_s: float = 0.0                          # predicted GPU seconds of its census
    device: tuple = field(default=None, repr=False)   # resident device copies (row_ptr, col)


class CensusServer:
    def __init__(self, budget_bytes: float = 120e9, workers: int = 2, max_batch: int = 512,
                 max_batch_edges: int = 20_000_000, max_batch_seconds: float = 0.25, run_batch=None, upload=None,
                 device=0, predictor: Predictor | None = None):
        self.budget = int(budget_bytes)
        self.max_batch_seconds = max_batch_seconds
        self.predictor = predictor or Predictor()
        self.batch_predictions: list[tuple[float, float]] = []   # (predicted, measured) seconds per batch
        self.in_use = 0
        self.pending_uploads = 0
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
        fut: Future = Future()
        if n < 0 or len(row_ptr) != n + 1 or (n > 0 and (row_ptr[0] != 0 or np.any(np.diff(row_ptr) < 0)
                                                          or row_ptr[-1] != len(col))):
            fut.set_exception(ValueError("malformed row pointer: row_ptr[0] = 0, non-decreasing, "
                                         "row_ptr[n] = len(col) required"))
            return fut
        m = int(row_ptr[-1]) // 2 if n > 0 else 0
        deg = np.diff(row_ptr) if n > 0 else np.zeros(0, np.int64)
        need = footprint_bytes(n, m, triangle_bound(row_ptr, col), int(deg.max()) if n > 0 else 0)
        req = Request(n, row_ptr, col, fut, time.perf_counter(), need)
        req.predicted_s = self.predictor.seconds(host_counts(row_ptr, col))
        if req.bytes > self.budget:
            fut.set_exception(MemoryError(f"request needs ~{req.bytes} B, budget is {self.budget} B"))
            return fut
        with self.lock:
            if self.closed:
                raise RuntimeError("server closed")
            self.waiting.append(req)
            reserved = self._reserve_locked()
        self._upload_reserved(reserved)
        return fut

    def close(self, wait: bool = True):
        with self.lock:
            self.closed = True
            self.lock.notify_all()
        if wait:
            for t in self.workers:
                t.join()

    # ------------------------------------------------------------------ internals
    def _reserve_locked(self):
        """Take the waiting requests that fit, FIFO (the head waits until it
        fits, later requests do not overtake it), and reserve their bytes.
        Their uploads happen outside the lock (_upload_reserved)."""
        reserved = []
        while self.waiting and self.in_use + self.waiting[0].bytes <= self.budget:
            req = self.waiting.popleft()
            self.in_use += req.bytes
            self.pending_uploads += 1
            req.t_admit = time.perf_counter()
            reserved.append(req)
        return reserved

    def _upload_reserved(self, reserved):
        """Copy reserved requests to the device without holding the lock, then
        hand them to the workers (or release their bytes if the copy failed)."""
        done = []
        for req in reserved:
            try:
                req.device = self._upload(req)
                done.append((req, None))
            except Exception as e:                       # upload failed: release and report
                done.append((req, e))
        if not done:
            return
        with self.lock:
            self.pending_uploads -= len(done)
            for req, err in done:
                if err is None:
                    self.admitted.append(req)
                else:
                    self.in_use -= req.bytes
            more = self._reserve_locked() if any(err is not None for _, err in done) else []
            self.lock.notify_all()
        for req, err in done:
            if err is not None:
                req.future.set_exception(err)
        self._upload_reserved(more)

    def _uploading(self) -> bool:
        """Some reserved request is still being copied to the device."""
        return self.pending_uploads > 0

    def _take_batch_locked(self):
        batch, edges, secs = [], 0, 0.0
        while self.admitted and len(batch) < self.max_batch:
            r = self.admitted[0]
            e = int(r.row_ptr[-1]) if r.n > 0 else 0
            if batch and (edges + e > self.max_batch_edges or secs + r.predicted_s > self.max_batch_seconds):
                break
            batch.append(self.admitted.popleft())
            edges += e
            secs += r.predicted_s
        return batch

    def _worker(self, k: int):
        stream = self._make_stream()
        while True:
            with self.lock:
                while not self.admitted and not (self.closed and not self.waiting and not self._uploading()):
                    self.lock.wait(timeout=0.05)
                if not self.admitted and self.closed and not self.waiting and not self._uploading():
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
                self.batch_predictions.append((sum(r.predicted_s for r in batch), t1 - t0))
                reserved = self._reserve_locked()
                self.lock.notify_all()
            self._upload_reserved(reserved)
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
        out = {"p50_ms": float(np.percentile(lat, 50)), "p99_ms": float(np.percentile(lat, 99)),
               "mean_ms": float(lat.mean()), "count": int(lat.size),
               "mean_batch": float(np.mean(self.batches)) if self.batches else 0.0}
        if self.batch_predictions:
            rel = [abs(p / m - 1.0) for p, m in self.batch_predictions if m > 0]
            out["predicted_vs_measured_batch_time_median_rel_err"] = float(np.median(rel)) if rel else None
        return out


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
