"""Benchmark: exact 34-class 5-vertex census (plus 3-/4-vertex counts) of one
synthetic graph per step, in edges per second.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--workload rmat22|chung_lu|er500|batch|serve]
  python bench.py --impl reference ...     # the CPU oracle, timed on a bounded sample

The default workload is the R-MAT scale-22 graph (~64.2M edges).  One step =
one escape_census5 call on a graph already resident in HBM (its CSR loaded
once before timing): orientation, every enumeration kernel and the 128-bit
assembly.  The L2 cache is flushed (256 MB write) between steps.  The
end-to-end figure (host CSR in pinned memory, load + census + result read
back) is timed over every step, or over three steps when a census takes a
second or more.
N > 1 (torchrun, NCCL) splits the census of the one graph over the ranks:
every rank counts the work items it owns (escape_census5_part), the ranks
add their sums and per-element arrays (the census's one exchange step,
paper_1610_09411_gb300/shard.py) and finish (strong scaling: value = the
graph's edges / the slowest rank's time per step).  One JSON line is printed
by rank 0.
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import threading
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "edges/s for full 34-class induced 5-vertex census"
UNIT = "edges/s"

WORKLOADS = {
    "chung_lu": "Chung-Lu power law n=262144, exponent 2.1, mean degree 16, max 8192, seed 1 (~2.0M edges)",
    "rmat22": "R-MAT scale 22, edge factor 16, (0.57,0.19,0.19,0.05), seed 1 (~64.2M edges)",
    "er500": "Erdos-Renyi G(500, 0.012), seed 0",
    "batch": "batch of graphs: sizes uniform 20-2000, half G(n,p) p~U(0.01,0.3), half BA m~U{2..6}, seed 2024",
    "serve": "Poisson stream of Chung-Lu (exponent 2.3, mean degree 16) requests, m log-uniform 1e3-5e6, "
             "120 GB admission budget",
}
# per-kernel algorithmic bytes: (phase, kernel, description, function of the oracle sums)
ALG_BYTES = {
    "wheels": ("k_wheels_cta / k_wheels_warp", "4 B x D (one id read per diamond, Thm 11 wheel sweep)",
               lambda s: 4 * s["D"]),
    "pairs": ("k_pairs", "4 B x (W + D) (one id read per wedge and per diamond, Thms 11-12; kernels "
              "k_pair_classify, k_pairs_hash<4096>, k_pairs_hash<16384>, k_pairs_win)",
              lambda s: 4 * (s["W"] + s["D"])),
    "cliques": ("k_clique_large / k_clique_warp", "4 B x (2 W++ + W+-) adjacency reads of the bit-matrix builds",
                lambda s: None),
    "cycles5": ("k_cycles5", "4 B x DP' (3-path endpoints)", lambda s: None),
}


def make_graph(name: str):
    import graphgen as gg
    if name == "chung_lu":
        return gg.config_chung_lu(1)
    if name == "rmat22":
        return gg.config_rmat(22, 1)
    if name == "er500":
        return gg.config_er500(0)
    raise SystemExit(f"unknown workload {name}")


def oracle_sums(name: str, g):
    """Counts the algorithmic-byte formulas need, as stored by the oracle
    (tests/golden: the whole census's sums, or W, T and D alone); None when no
    stored result matches this graph."""
    sys.path.insert(0, os.path.join(ROOT, "tests"))
    try:
        from gpu_util import graph_hash
        for kind in ("census", "sums"):
            path = os.path.join(ROOT, "tests", "golden", f"{kind}_{name}.json")
            if not os.path.exists(path):
                continue
            with open(path) as f:
                gold = json.load(f)
            if gold["sha256"] != graph_hash(g):
                continue
            return {k: int(v) for k, v in gold["sums"].items()}
    except Exception:
        pass
    return None


def measured_peak():
    path = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(path) as f:
            p = json.load(f)
        return float(p["hbm_gbs"]), "measured"
    except Exception:
        return 6800.0, "fallback"


class ClockSampler:
    """nvidia-smi clock/throttle samples during the timed region."""

    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        try:
            fd, self.path = tempfile.mkstemp(suffix=".csv")
            os.close(fd)
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "200"], stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        rows = []
        with open(self.path) as f:
            for line in f:
                parts = [x.strip() for x in line.split(",")]
                if len(parts) >= 9:
                    rows.append(parts)
        os.unlink(self.path)
        if not rows:
            return None
        def num(x):
            try:
                return float(x)
            except ValueError:
                return None
        sm = [num(r[1]) for r in rows if num(r[1]) is not None]
        smax = [num(r[2]) for r in rows if num(r[2]) is not None]
        reasons = set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            for k, name in enumerate(names):
                if r[5 + k].lower() == "active":
                    reasons.add(name)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(rows)}


# the code that decides each swept phase's DRAM traffic: a section of
# census.cu between two of its banner comments, and the host lines that shape
# its launches
DIGEST_SECTIONS = {
    "k_pairs": ([("// Thm 11/12: N13", "// Thm 11: N18 (wheels)"),
                 ("struct PairPlan {", "\ncudaError_t run_census(")],
                ("PAIR_", "PairPlan", "pplan", "plan_pair", "launch_pairs", "k_pairs", "ptasks", "tsB", "pwin")),
}


def source_digest(kernel: str = "k_pairs") -> str:
    """Digest of what decides a kernel's DRAM traffic: the section of
    census.cu that holds the kernel and its device helpers, the counter struct
    it uses and every line naming its constants or launch configuration.
    Edits elsewhere leave it unchanged; any edit of the kernel changes it (and
    a failed extraction hashes the whole file, which only makes a stored figure
    look stale)."""
    path = os.path.join(ROOT, "paper_1610_09411_gb300", "csrc", "census.cu")
    with open(path) as f:
        src = f.read()
    h = hashlib.sha256()
    spans, keys = DIGEST_SECTIONS.get(kernel, ([(f" {kernel}(", "\n}\n")], (kernel,)))
    spans = spans + [("struct TaggedCounters {", "\n};\n")]
    cut = []
    for begin, end in spans:
        a = src.find(begin)
        b = src.find(end, a + 1) if a >= 0 else -1
        if min(a, b) < 0:
            h.update(src.encode())
            return h.hexdigest()[:16]
        cut.append((a, b))
    rest, pos = [], 0
    for a, b in sorted(cut):
        h.update(src[a:b].encode())
        rest.append(src[pos:a])
        pos = max(pos, b)
    rest.append(src[pos:])
    for line in "".join(rest).splitlines():
        if any(k in line for k in keys):
            h.update(line.encode())
    return h.hexdigest()[:16]


def stored_traffic(kernel: str, workload: str):
    """DRAM bytes per launch from the committed ncu summary, if it was taken on
    the current kernel source."""
    path = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        with open(path) as f:
            t = json.load(f)
        rec = t.get(f"{kernel}:{workload}")
        if rec and rec.get("source_sha") == source_digest(kernel.split(" ")[0]):
            return rec["dram_bytes_per_launch"]
    except Exception:
        pass
    return None


# bounded samples of each workload for the oracle's CPU timings: the same
# generator and parameters at fewer vertices (cpu_baseline: ~10-30 s of one
# core; reference arm: a few seconds per step)
SAMPLES = {
    "chung_lu": {"baseline": ("Chung-Lu n=32768 (exponent 2.1, mean 16, clip 8192, seed 1)",
                              lambda gg: gg.chung_lu(32768, 2.1, 16.0, 8192.0, 1)),
                 "reference": ("Chung-Lu n=8192 (exponent 2.1, mean 16, clip 8192, seed 1)",
                               lambda gg: gg.chung_lu(8192, 2.1, 16.0, 8192.0, 1))},
    "rmat22": {"baseline": ("R-MAT scale 14, edge factor 16, (0.57,0.19,0.19,0.05), seed 1",
                            lambda gg: gg.config_rmat(14, 1)),
               "reference": ("R-MAT scale 12, edge factor 16, (0.57,0.19,0.19,0.05), seed 1",
                             lambda gg: gg.config_rmat(12, 1))},
    "er500": {"baseline": ("Erdos-Renyi G(500, 0.012), seed 0", lambda gg: gg.config_er500(0)),
              "reference": ("Erdos-Renyi G(500, 0.012), seed 0", lambda gg: gg.config_er500(0))},
}


# workloads without a stored full census, and the stored run of the same
# generator at a smaller size reported beside their CPU baseline
RELATED_FULL = {"rmat22": ("rmat20", "R-MAT scale 20 (the same generator and parameters, 15.7M edges)")}


def stored_oracle_run(name: str):
    """Wall time, thread count and host of the stored oracle result of the full
    workload graph (tests/golden), or None."""
    path = os.path.join(ROOT, "tests", "golden", f"census_{name}.json")
    try:
        with open(path) as f:
            gold = json.load(f)
        return {"seconds": gold["oracle_seconds"], "threads": gold.get("oracle_threads", 1),
                "host": gold.get("oracle_host", "the build container"), "m": gold["m"]}
    except Exception:
        return None


def cpu_baseline(workload: str):
    """The oracle as it stands (serial build), on a bounded sample of the
    workload, plus the stored full-graph oracle run for comparison."""
    import graphgen as gg
    import oracle
    desc, make = SAMPLES.get(workload, SAMPLES["chung_lu"])["baseline"]
    g = make(gg)
    oracle.build()
    t0 = time.perf_counter()
    oracle.census(g)
    dt = time.perf_counter() - t0
    out = {"value": g.m / dt, "unit": UNIT, "cores": 1, "kind": "oracle",
           "sample": f"{desc}, m={g.m}, full census, {dt:.1f} s on one core"}
    full = stored_oracle_run(workload)
    if full:
        out["full_graph"] = {"value": full["m"] / full["seconds"], "unit": UNIT, "seconds": full["seconds"],
                             "threads": full["threads"], "host": full["host"],
                             "note": "the stored oracle result of the whole workload graph (tests/golden)"}
    elif workload in RELATED_FULL:
        name, what = RELATED_FULL[workload]
        rel = stored_oracle_run(name)
        if rel:
            out["related_full_graph"] = {"value": rel["m"] / rel["seconds"], "unit": UNIT, "seconds": rel["seconds"],
                                         "m": rel["m"], "threads": rel["threads"], "host": rel["host"],
                                         "note": f"the stored oracle result of {what} (tests/golden); the whole "
                                                 "workload graph has no stored full census"}
    return out


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    import graphgen as gg
    import oracle
    oracle.build()
    desc, make = SAMPLES.get(args.workload, SAMPLES["chung_lu"])["reference"]
    g = make(gg)
    for _ in range(args.warmup):
        oracle.census(g)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.census(g)
    dt = time.perf_counter() - t0
    value = g.m * args.steps / dt
    line = {
        "impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1000 * dt / args.steps,
        "higher_is_better": True, "scaling": "strong", "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "sample": f"{desc} per step"},
        "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                         "sample": f"{desc}, m={g.m}, full census per step (serial oracle build)"},
        "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }
    print(json.dumps(line), flush=True)


def census_alg_bytes(g, sums):
    """Algorithmic bytes of the whole census, 4 B per vertex id the method must
    read plus 8 B per count-array entry: the orientation (2m), the triangle
    intersections (sum over oriented edges u->v of d+(u) + d+(v)), both 4-cycle
    passes (2 (W++ + W+-)), the pair sweep (W), the cc and wheel sweeps (2D)
    and the directed 3-paths of the 5-cycle count (DP), with W and D from the
    stored oracle result and the rest from the degree-ordered DAG.  The 4-clique
    and bipyramid terms need per-triangle counts that are not stored, so this
    is a lower bound of the full formula."""
    import numpy as np
    deg = g.degrees().astype(np.int64)
    n = g.n
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    dst = g.col.astype(np.int64)
    up = (deg[src] < deg[dst]) | ((deg[src] == deg[dst]) & (src < dst))      # src precedes dst
    dplus = np.bincount(src[up], minlength=n).astype(np.int64)
    dminus = deg - dplus
    wpp = int((dplus * (dplus - 1) // 2).sum())
    wpm = int((dplus * dminus).sum())
    tri = int((dplus[src[up]] + dplus[dst[up]]).sum())
    dp = int(((dplus[src[up]] - 1) * dplus[dst[up]]).sum())                 # i <- a -> b -> j
    terms = {"orient": 2 * g.m, "triangles": tri, "cycles4": 2 * (wpp + wpm), "pairs": sums["W"],
             "cc_wheels": 2 * sums["D"], "paths3": dp}
    total = 4 * sum(terms.values()) + 8 * (n + 3 * g.m)
    return total, {k: int(v) for k, v in terms.items()}


def slowest_rank_ms(total_ms: float, world: int, device: str) -> float:
    """Max over ranks of the timed region (the job ends with the slowest rank)."""
    if world <= 1:
        return total_ms
    import torch
    import torch.distributed as dist
    t = torch.tensor([total_ms], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    dist.barrier()
    return float(t.item())


def job_value(m: int, ms_per_step: float) -> float:
    """Whole-job edges/s: the ranks together count one graph of m edges per step."""
    return m / (ms_per_step / 1000.0)


def _pack(graphs):
    import numpy as np
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    rps, cols, base = [], [], 0
    for k, g in enumerate(graphs):
        voff[k + 1] = voff[k] + g.n
        rps.append(g.row_ptr[:-1] + base)
        cols.append(g.col)
        base += g.nnz
    rp = np.concatenate(rps + [np.array([base])]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32)
    return voff, rp, col


def run_batch_bench(args):
    """Batched census: one fused escape_census5_batch call per step over the
    whole batch (resident on the device) vs one escape_census5 call per graph."""
    import torch
    import graphgen as gg
    torch.cuda.set_device(0)
    from paper_1610_09411_gb300 import build as pbuild
    pbuild.build()
    from paper_1610_09411_gb300 import escape as esc
    graphs = gg.batch_graphs(args.batch_count, 2024)
    edges = sum(g.m for g in graphs)
    voff, rp, col = _pack(graphs)
    dv, dr, dc = (torch.from_numpy(x).cuda() for x in (voff, rp, col))
    torch.cuda.synchronize()
    for _ in range(args.warmup):
        res = esc.escape_census5_batch(dv, dr, dc)
    stream = torch.cuda.current_stream()
    total = 0.0
    for _ in range(args.steps):
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = esc.escape_census5_batch(dv, dr, dc)
        e1.record(stream)
        e1.synchronize()
        total += e0.elapsed_time(e1)
    ms = total / args.steps
    # one launch sequence per graph (each graph resident on the device)
    handles = [esc.escape_load_csr(g.n, torch.from_numpy(g.row_ptr).cuda(), torch.from_numpy(g.col).cuda())
               for g in graphs]
    torch.cuda.synchronize()
    t0 = time.perf_counter()
    single = [esc.escape_census5(h) for h in handles]
    torch.cuda.synchronize()
    ms_single = 1000 * (time.perf_counter() - t0)
    for h in handles:
        esc.escape_free(h)
    same = all(a == b for a, b in zip(res, single))
    line = {"metric": "batched graphs/s (full census per graph)", "value": len(graphs) / (ms / 1000.0),
            "unit": "graphs/s", "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "u128", "data": "synthetic",
            "config": {"workload": WORKLOADS["batch"], "graphs": len(graphs), "edges": edges},
            "edges_per_s": edges / (ms / 1000.0),
            "one_graph_per_launch": {"graphs_per_s": len(graphs) / (ms_single / 1000.0), "ms": ms_single},
            "speedup_vs_one_graph_per_launch": ms_single / ms, "results_identical": same}
    print(json.dumps(line), flush=True)


def run_serve_bench(args):
    """Serving: Poisson arrivals at each rate, continuous batching over three
    streams vs the one-at-a-time path (one worker, batches of one)."""
    import numpy as np
    import torch
    import graphgen as gg
    torch.cuda.set_device(0)
    from paper_1610_09411_gb300 import build as pbuild
    pbuild.build()
    from paper_1610_09411_gb300 import escape as esc  # noqa: F401
    from paper_1610_09411_gb300.serve import CensusServer, poisson_arrivals, replay
    rng_seed = 31
    graphs = []
    for k in range(args.serve_requests):
        u = (gg.stream_draw(rng_seed, 9, k) >> 11) / float(1 << 53)
        m_target = 10 ** (3 + u * (np.log10(5e6) - 3))
        n = max(64, int(m_target / 8))
        graphs.append(gg.chung_lu(n, 2.3, 16.0, max(16.0, min(8192.0, n / 4)), gg.stream_draw(rng_seed, 10, k)))
    edges = sum(g.m for g in graphs)
    # warm up the library on a small graph
    g0 = gg.erdos_renyi(100, 0.1, 1)
    esc.census(g0.row_ptr, g0.col, n=g0.n)
    out = {"metric": "served census: p50/p99 latency and edges/s", "unit": "ms", "higher_is_better": False,
           "n_gpus": 1, "dtype": "u128", "data": "synthetic",
           "config": {"workload": WORKLOADS["serve"], "requests": len(graphs), "edges": edges,
                      "workers": 3}, "rates": {}}
    for rate in [float(r) for r in args.serve_rates.split(",")]:
        arr = poisson_arrivals(rate, len(graphs), 7)
        row = {}
        for mode, kw in (("continuous_batching", dict(workers=3)),
                         ("one_at_a_time", dict(workers=1, max_batch=1))):
            srv = CensusServer(budget_bytes=120e9, **kw)
            try:
                t0 = time.perf_counter()
                futs = replay(srv, graphs, arr)
                for f in futs:
                    f.result()
                span = time.perf_counter() - t0
            finally:
                srv.close()
            st = srv.latency_stats()
            st["edges_per_s"] = edges / span
            st["makespan_s"] = span
            row[mode] = st
        out["rates"][str(int(rate))] = row
    best = out["rates"][max(out["rates"], key=lambda r: float(r))]["continuous_batching"]
    out["value"] = best["p99_ms"]
    print(json.dumps(out), flush=True)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=None,
                    help="timed steps (default: 3 for the R-MAT 22 census, about a minute; 5 otherwise)")
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="rmat22", choices=sorted(WORKLOADS))
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--batch-count", type=int, default=1000, help="graphs in the batch workload (config: 10000)")
    ap.add_argument("--serve-requests", type=int, default=64)
    ap.add_argument("--serve-rates", default="100,1000,10000")
    args = ap.parse_args()
    if args.steps is None:
        args.steps = 3 if args.workload == "rmat22" else 5
    if args.warmup < 3:
        args.warmup = 3
    if args.impl == "reference":
        return run_reference(args)
    if args.workload == "batch":
        return run_batch_bench(args)
    if args.workload == "serve":
        return run_serve_bench(args)

    import numpy as np
    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    from paper_1610_09411_gb300 import build as pbuild
    if rank == 0 or world == 1:
        pbuild.build()
    if world > 1:
        dist.barrier()
    from paper_1610_09411_gb300 import autotune, escape as esc
    from paper_1610_09411_gb300 import shard

    g = make_graph(args.workload)
    knobs = autotune.apply(g.nnz)               # the tuned launch knobs of the graph's size class
    cps = autotune.cta_per_sm()

    def census_step(handle):
        if world == 1:
            return esc.escape_census5(handle)
        return shard.sharded_census(handle, g.n, g.nnz)
    stream = torch.cuda.current_stream()
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    torch.cuda.synchronize()
    h = esc.escape_load_csr(g.n, rp, col)
    esc.escape_set_options(h, False, cps, None)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.int32, device="cuda")
    for _ in range(args.warmup):
        res = census_step(h)

    sampler = ClockSampler(local) if rank == 0 else None
    phase_tot = {}
    launches = 0
    total_ms = 0.0
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    if sampler:
        sampler.start()
    for _ in range(args.steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        res = census_step(h)
        e1.record(stream)
        e1.synchronize()
        total_ms += e0.elapsed_time(e1)
        if world == 1:
            for k, v in esc.escape_last_phase_ms(h).items():
                phase_tot[k] = phase_tot.get(k, 0.0) + v
        launches += esc.escape_last_kernel_launches(h)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks = sampler.stop() if sampler else None
    # outside the timed region: one census with the phases run one after
    # another, for each kernel's duration alone
    alone_phase = {}
    if world == 1:
        esc.escape_set_options(h, False, cps, True)
        esc.escape_census5(h)
        alone_phase = esc.escape_last_phase_ms(h)
        esc.escape_set_options(h, False, cps, None)
    total_ms = slowest_rank_ms(total_ms, world, "cuda")
    ms_per_step = total_ms / args.steps
    value = job_value(g.m, ms_per_step)

    # end to end through the public C ABI with pinned host buffers: H2D of the
    # CSR, the census, D2H of the result struct, every step
    hrp = torch.from_numpy(g.row_ptr).pin_memory()
    hcol = torch.from_numpy(g.col).pin_memory()
    h2d = int(g.row_ptr.nbytes + g.col.nbytes)
    d2h = 2 * 49 * 16
    e2e_ms = 0.0
    # graphs of a second or more per census: a few end-to-end steps suffice
    e2e_steps = args.steps if ms_per_step < 1000 else min(args.steps, 3)
    for _ in range(e2e_steps):
        flush.fill_(1)
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        hh = esc.escape_load_csr(g.n, hrp.numpy(), hcol.numpy())
        esc.escape_set_options(hh, False, cps, None)
        r2 = census_step(hh)
        esc.escape_free(hh)
        e2e_ms += 1000 * (time.perf_counter() - t0)
        assert r2["c5"] == res["c5"]
    e2e_ms = slowest_rank_ms(e2e_ms, world, "cuda")
    e2e_value = g.m / (e2e_ms / e2e_steps / 1000.0)
    esc.escape_free(h)

    if rank != 0:
        if world > 1:
            dist.barrier()
            dist.destroy_process_group()
        return

    # roofline of the dominant kernel: the phase with a byte model that takes
    # longest when every phase runs alone (the ranking of the serialised ncu
    # launch list; overlapped spans inflate the side-stream phases)
    sums = oracle_sums(args.workload, g)
    avg_phase = {k: v / args.steps for k, v in phase_tot.items()}
    roof = None
    cand = [(alone_phase.get(p, 0.0) or avg_phase.get(p, 0.0), p) for p in ALG_BYTES]
    cand.sort(reverse=True)
    peak, peak_src = measured_peak()
    for _, phase in cand:
        kernel, desc, fn = ALG_BYTES[phase]
        ms = avg_phase.get(phase, 0.0)
        if sums is None or ms <= 0:
            continue
        b = fn(sums)
        if b is None:
            continue
        achieved = b / (ms / 1000.0) / 1e9
        alone = alone_phase.get(phase, 0.0)
        roof = {"bound": "hbm", "achieved": achieved, "peak": peak, "unit": "GB/s", "frac": achieved / peak,
                "traffic": stored_traffic(kernel, args.workload), "kernel": kernel, "phase_ms": ms,
                "algorithmic_bytes": b, "bytes_model": desc, "peak_source": f"{peak_src} hbm_gbs",
                "achieved_alone": (b / (alone / 1000.0) / 1e9) if alone > 0 else None,
                "note": "phase_ms is timed with the independent sweeps overlapping on side streams; "
                        "achieved_alone uses the phase's time when every phase runs alone"}
        break
    census_roof = None
    if sums is not None:
        b_all, terms = census_alg_bytes(g, sums)
        ach = b_all / (ms_per_step / 1000.0) / 1e9
        census_roof = {"bound": "hbm", "achieved": ach, "peak": peak, "unit": "GB/s", "frac": ach / peak,
                       "algorithmic_bytes": b_all, "terms": terms,
                       "bytes_model": "4 B x (2m + sum_{u->v}(d+u + d+v) + 2(W++ + W+-) + W + 2D + DP) + "
                                      "8 B x (n + 3m); 4-clique and bipyramid terms omitted (lower bound)"}
    cpu = None if args.no_cpu_baseline else cpu_baseline(args.workload)
    line = {
        "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": ms_per_step, "higher_is_better": True, "scaling": "strong",
        "vs_baseline": None, "dtype": "u128", "data": "synthetic",
        "config": {"workload": WORKLOADS[args.workload], "n": g.n, "m": g.m,
                   "l2": "flushed between steps (256 MB write)",
                   "tuning": knobs or "library defaults",
                   "parallelism": f"one census split over {world} GPUs (owned items, one exchange)"
                                  if world > 1 else "1 GPU"},
        "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
                "steps": e2e_steps},
        "gpu_launches": launches,
        "phase_ms": {k: round(v, 3) for k, v in avg_phase.items()},
        "phase_ms_alone": {k: round(v, 3) for k, v in alone_phase.items()},
        "roofline": roof,
        "census_roofline": census_roof,
        "cpu_baseline": cpu,
        "clocks": clocks,
    }
    print(json.dumps(line), flush=True)
    if world > 1:
        dist.barrier()
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
