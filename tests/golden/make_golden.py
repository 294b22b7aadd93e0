"""Write stored oracle results for the larger workloads (run from the repo root).

Calls only the seeded generators and oracle/; every value written here comes
from the CPU oracle.  Each file records a SHA-256 of the generated CSR so a
test can tell whether the graph it regenerates is the one the values were
computed for (and recompute them live if not).

    python tests/golden/make_golden.py chung_lu er500 two_hubs
    python tests/golden/make_golden.py --parallel rmat20 batch24
    python tests/golden/make_golden.py --elements rmat22
    python tests/golden/make_golden.py --parallel --sums rmat22
    python tests/golden/make_golden.py --parallel --pairs rmat22
    python tests/golden/make_golden.py --parallel --cliques rmat22
    python tests/golden/make_golden.py --parallel --cliques5 rmat22

--parallel runs the OpenMP build of the same oracle source on OMP_NUM_THREADS
threads (its equality with the serial build is pinned in test_oracle_pins).
"""
import json
import os
import platform
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, os.path.dirname(os.path.dirname(HERE)))
sys.path.insert(0, os.path.dirname(HERE))

import graphgen as gg  # noqa: E402
import oracle  # noqa: E402
from gpu_util import graph_hash  # noqa: E402


WORKLOADS = {
    "chung_lu": lambda: gg.config_chung_lu(1),
    "er500": lambda: gg.config_er500(0),
    "two_hubs": lambda: gg.two_hubs(),
    "batch24": lambda: gg.batch_member(24, 2024),        # G(1250, 0.279): a dense member of the batch workload
    "rmat20": lambda: gg.config_rmat(20, 1),
    "rmat22": lambda: gg.config_rmat(22, 1),
}


def element_sample(g, seed=2024, k=40, hubs=10):
    """Vertices and edges whose per-element values are stored: the `hubs`
    highest-degree vertices, their mutual edges and first entries, and `k`
    seeded random vertices (degree >= 1) and edges."""
    import numpy as np
    deg = g.degrees()
    rng = np.random.default_rng(seed)
    top = [int(v) for v in np.argsort(-deg, kind="stable")[:hubs]]
    nz = np.nonzero(deg > 0)[0]
    rand_v = [int(v) for v in rng.choice(nz, size=min(k, nz.size), replace=False)] if nz.size else []
    verts = sorted(set(top) | set(rand_v))
    slots = set(int(p) for p in rng.choice(g.nnz, size=min(k, g.nnz), replace=False)) if g.nnz else set()
    for u in top:
        row = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        for j in range(min(4, row.size)):
            slots.add(int(g.row_ptr[u] + j))
        for v in top:
            q = np.searchsorted(row, v)
            if q < row.size and row[q] == v:
                slots.add(int(g.row_ptr[u] + q))
    slots = sorted(slots)
    src = np.repeat(np.arange(g.n), deg)
    return verts, [(int(src[p]), int(g.col[p])) for p in slots], slots


def write(name, parallel=False):
    g = WORKLOADS[name]()
    t0 = time.time()
    c = oracle.census(g, per_element=True, parallel=parallel)
    pe = c["per_element"]
    verts, edges, slots = element_sample(g)
    out = {
        "workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.num_threads(parallel),
        "oracle_host": f"{platform.machine()}, {os.cpu_count()} cores",
        "c3": [str(x) for x in c["c3"]], "c4": [str(x) for x in c["c4"]], "c5": [str(x) for x in c["c5"]],
        "n3": [str(x) for x in c["n3"]], "n4": [str(x) for x in c["n4"]], "n5": [str(x) for x in c["n5"]],
        "sums": {k: str(v) for k, v in c["sums"].items()},
        "elements": {
            "vertices": verts, "edges": edges,
            **{key: [str(int(pe[key][v])) for v in verts] for key in ("t_i", "C4_i", "K4_i")},
            **{key: [str(int(pe[key][p])) for p in slots] for key in ("T_e", "C4_e", "K4_e")},
        },
    }
    with open(os.path.join(HERE, f"census_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["oracle_seconds"], "s")


def write_elements(name):
    """Per-element values of the sampled vertices and edges (the highest-degree
    vertices among them) from their definitions alone (oracle.vertex_elements,
    oracle.edge_elements), for graphs whose full oracle census takes too long."""
    import numpy as np
    g = WORKLOADS[name]()
    t0 = time.time()
    verts, edges, slots = element_sample(g)
    v = oracle.vertex_elements(g, verts)
    e = oracle.edge_elements(g, np.array([a for a, _ in edges]), np.array([b for _, b in edges]))
    out = {
        "workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
        "oracle_seconds": round(time.time() - t0, 1),
        "elements": {
            "vertices": verts, "edges": edges,
            "t_i": [str(int(x)) for x in v["t_i"]], "C4_i": [str(int(x)) for x in v["C4_i"]],
            "T_e": [str(int(x)) for x in e["T_e"]], "K4_e": [str(int(x)) for x in e["K4_e"]],
            "C4_e": [str(int(x)) for x in e["C4_e"]],
        },
    }
    with open(os.path.join(HERE, f"elements_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "elements", out["oracle_seconds"], "s")


def write_sums(name, parallel=False):
    """W, T and D of a workload from their definitions (oracle.wedge_diamond_sums):
    the unit counts of the benchmark's byte model where the full census is out of reach."""
    g = WORKLOADS[name]()
    t0 = time.time()
    w = oracle.wedge_diamond_sums(g, parallel=parallel)
    out = {"workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
           "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.num_threads(parallel),
           "oracle_host": f"{platform.machine()}, {os.cpu_count()} cores",
           "sums": {k: str(v) for k, v in w.items()}}
    with open(os.path.join(HERE, f"sums_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "sums", out["oracle_seconds"], "s")


def write_pairs(name, parallel=False):
    """C4 and N13 (non-induced K2,3) of a workload from the two-hop pair counts
    alone (oracle.pair_sums), where the full census is out of reach."""
    g = WORKLOADS[name]()
    t0 = time.time()
    w = oracle.pair_sums(g, parallel=parallel)
    out = {"workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
           "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.num_threads(parallel),
           "oracle_host": f"{platform.machine()}, {os.cpu_count()} cores",
           "sums": {k: str(v) for k, v in w.items()}}
    with open(os.path.join(HERE, f"pairs_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "pairs", out["oracle_seconds"], "s")


def write_cliques(name, parallel=False):
    """The 4-clique count of a workload alone (oracle.clique4_count), where the
    full census is out of reach."""
    g = WORKLOADS[name]()
    t0 = time.time()
    k4 = oracle.clique4_count(g, parallel=parallel)
    out = {"workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
           "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.num_threads(parallel),
           "oracle_host": f"{platform.machine()}, {os.cpu_count()} cores",
           "sums": {"K4": str(k4)}}
    with open(os.path.join(HERE, f"cliques_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "cliques", out["oracle_seconds"], "s")


def write_cliques5(name, parallel=False):
    """The 5-clique count of a workload alone (oracle.clique5_count), where the
    full census is out of reach."""
    g = WORKLOADS[name]()
    t0 = time.time()
    k5 = oracle.clique5_count(g, parallel=parallel)
    out = {"workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
           "oracle_seconds": round(time.time() - t0, 1), "oracle_threads": oracle.num_threads(parallel),
           "oracle_host": f"{platform.machine()}, {os.cpu_count()} cores",
           "sums": {"K5": str(k5)}}
    with open(os.path.join(HERE, f"cliques5_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, "cliques5", out["oracle_seconds"], "s")


if __name__ == "__main__":
    par = "--parallel" in sys.argv
    names = [a for a in sys.argv[1:] if not a.startswith("--")]
    for name in names or ["chung_lu", "er500", "two_hubs"]:
        if "--elements" in sys.argv:
            write_elements(name)
        elif "--sums" in sys.argv:
            write_sums(name, par)
        elif "--pairs" in sys.argv:
            write_pairs(name, par)
        elif "--cliques5" in sys.argv:
            write_cliques5(name, par)
        elif "--cliques" in sys.argv:
            write_cliques(name, par)
        else:
            write(name, par)
