"""Write stored oracle results for the larger workloads (run from the repo root).

Calls only the seeded generators and oracle/; every value written here comes
from the CPU oracle.  Each file records a SHA-256 of the generated CSR so a
test can tell whether the graph it regenerates is the one the values were
computed for (and recompute them live if not).

    python tests/golden/make_golden.py chung_lu er500 two_hubs
    python tests/golden/make_golden.py --parallel rmat20 rmat22

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
    "rmat20": lambda: gg.config_rmat(20, 1),
    "rmat22": lambda: gg.config_rmat(22, 1),
}


def write(name, parallel=False):
    g = WORKLOADS[name]()
    t0 = time.time()
    c = oracle.census(g, parallel=parallel)
    out = {
        "workload": name, "graph": g.name, "n": g.n, "m": g.m, "sha256": graph_hash(g),
        "oracle_seconds": round(time.time() - t0, 1),
        "oracle_threads": oracle.num_threads(parallel),
        "oracle_host": f"{platform.machine()}, {os.cpu_count()} cores",
        "c3": [str(x) for x in c["c3"]], "c4": [str(x) for x in c["c4"]], "c5": [str(x) for x in c["c5"]],
        "n3": [str(x) for x in c["n3"]], "n4": [str(x) for x in c["n4"]], "n5": [str(x) for x in c["n5"]],
        "sums": {k: str(v) for k, v in c["sums"].items()},
    }
    with open(os.path.join(HERE, f"census_{name}.json"), "w") as f:
        json.dump(out, f, indent=1)
    print(name, out["oracle_seconds"], "s")


if __name__ == "__main__":
    par = "--parallel" in sys.argv
    names = [a for a in sys.argv[1:] if not a.startswith("--")]
    for name in names or ["chung_lu", "er500", "two_hubs"]:
        write(name, par)
