"""Project-written autotuner for the census's launch knobs.

The knobs are environment variables the library reads when it plans a census
(results never depend on them, only the time does):

  ESC_PAIR_WINDOW     heavy pair-sweep items: 3 (the default) count every rank in
                      successive shared-memory windows; 2 one window over the top
                      ranks, tagged global counters below it; 1 no window
  ESC_PAIR_CLUSTER    CTAs per cluster for the heavy pair-sweep items (1, 2, 4, 8, 16;
                      the window needs 1)
  ESC_PAIR_SHAPE      heavy pair kernel: 1 = 512 threads x 3 CTAs per SM,
                      2 = 512 x 2, 3 = 1024 x 1
  ESC_WHEEL_WARP_MAX  wheel centres of at most this degree are split into warp
                      items, larger ones into CTA items (at most 1024)
  ESC_CLQ_WARP_DIN    clique items with d+ <= 32 and at most this many
                      in-neighbours are counted by one warp (at most 512)
  ESC_CTA_PER_SM      persistent CTAs per SM of the 4-cycle, 5-cycle and list
                      sweeps (escape_set_options; 1..4)

Graphs fall into size classes by their adjacency entries (2m).  tune() runs
coordinate descent on one representative graph of a class: each knob in turn
over its values, keeping the fastest (CUDA-event time of the census, best of
`reps`), and stores {class: {knob: value, "ms": best}} in tuning.json beside
this file.  apply(nnz) sets the stored knobs of a graph's class in the process
environment before a census; the bench calls it.

    python -m paper_1610_09411_gb300.autotune            # tune every class (GPU)
    python -m paper_1610_09411_gb300.autotune rmat22     # one class's representative
"""
from __future__ import annotations

import json
import os
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
TUNING_PATH = os.path.join(HERE, "tuning.json")

KNOBS = {
    "ESC_PAIR_WINDOW": [3, 2, 1],
    "ESC_PAIR_CLUSTER": [1, 2, 4, 8],
    "ESC_PAIR_SHAPE": [3, 2, 1],
    "ESC_WHEEL_WARP_MAX": [1024, 512, 256],
    "ESC_CLQ_WARP_DIN": [512, 256, 128],
    "ESC_CTA_PER_SM": [2, 3, 1, 4],
}
# upper bounds (exclusive) of 2m for the classes
CLASSES = [("small", 1 << 18), ("medium", 1 << 22), ("large", 1 << 25), ("huge", 1 << 62)]


def size_class(nnz: int) -> str:
    for name, hi in CLASSES:
        if nnz < hi:
            return name
    return CLASSES[-1][0]


def load(path: str = TUNING_PATH) -> dict:
    try:
        with open(path) as f:
            return json.load(f)
    except (OSError, ValueError):
        return {}


def apply(nnz: int, table: dict | None = None) -> dict:
    """Set (or clear) the tuned knobs of the class of a graph with nnz
    adjacency entries; returns the knobs set."""
    table = load() if table is None else table
    knobs = {k: v for k, v in table.get(size_class(nnz), {}).items() if k in KNOBS}
    for k in KNOBS:
        if k in knobs:
            os.environ[k] = str(knobs[k])
        else:
            os.environ.pop(k, None)
    return knobs


def cta_per_sm() -> int:
    """The tuned persistent-CTA count, or 0 (the library's default)."""
    try:
        return int(os.environ.get("ESC_CTA_PER_SM", "0"))
    except ValueError:
        return 0


def _time_census(h, reps: int) -> float:
    import torch
    from . import escape as esc
    esc.escape_set_options(h, False, cta_per_sm(), None)
    best = None
    for _ in range(reps):
        st = torch.cuda.current_stream()
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        esc.escape_census5(h)
        e1.record(st)
        e1.synchronize()
        ms = e0.elapsed_time(e1)
        best = ms if best is None else min(best, ms)
    return best


def tune(g, reps: int = 2, knobs=None, log=print) -> dict:
    """Coordinate descent over the knobs on graph g; returns {knob: value, "ms": best}."""
    import torch
    from . import escape as esc
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    torch.cuda.synchronize()
    h = esc.escape_load_csr(g.n, rp, col)
    knobs = knobs or list(KNOBS)
    try:
        best = {k: KNOBS[k][0] for k in knobs}
        for k in KNOBS:
            os.environ.pop(k, None)
        for k, v in best.items():
            os.environ[k] = str(v)
        esc.escape_census5(h)                                   # warm-up
        best_ms = _time_census(h, reps)
        ref = esc.escape_census5(h)
        for k in knobs:
            for v in KNOBS[k][1:]:
                os.environ[k] = str(v)
                ms = _time_census(h, reps)
                assert esc.escape_census5(h) == ref, "a launch knob changed the counts"
                log(f"{g.name} {k}={v}: {ms:.2f} ms (best {best_ms:.2f} ms with {best})")
                if ms < best_ms:
                    best_ms, best[k] = ms, v
            os.environ[k] = str(best[k])
    finally:
        esc.escape_free(h)
        for k in KNOBS:
            os.environ.pop(k, None)
    out = dict(best)
    out["ms"] = best_ms
    return out


def representatives():
    import graphgen as gg
    return {
        "small": lambda: gg.erdos_renyi(800, 0.15, 3),          # a dense batch-like member, 9.6e4 entries
        "medium": lambda: gg.config_chung_lu(1),                # 3.9e6 entries
        "large": lambda: gg.config_rmat(20, 1),                 # 3.1e7 entries
        "huge": lambda: gg.config_rmat(22, 1),                  # 1.3e8 entries
    }


def main(argv):
    root = os.path.dirname(HERE)
    if root not in sys.path:
        sys.path.insert(0, root)
    import torch
    torch.cuda.set_device(0)
    reps = {"small": 3, "medium": 3, "large": 2, "huge": 1}
    names = [a for a in argv if not a.startswith("-")] or [c for c, _ in CLASSES]
    table = load()
    for name in names:
        g = representatives()[name]()
        assert size_class(g.nnz) == name, (name, g.nnz)
        knobs = None
        if name == "huge":        # a census takes ~30 s here: the knobs that move it
            knobs = ["ESC_PAIR_WINDOW", "ESC_PAIR_CLUSTER", "ESC_PAIR_SHAPE", "ESC_WHEEL_WARP_MAX"]
        t0 = time.time()
        table[name] = tune(g, reps[name], knobs)
        table[name]["graph"] = g.name
        table[name]["tuning_s"] = round(time.time() - t0, 1)
        with open(TUNING_PATH, "w") as f:
            json.dump(table, f, indent=1)
        print(name, table[name], flush=True)


if __name__ == "__main__":
    main(sys.argv[1:])
