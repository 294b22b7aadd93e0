"""The stored oracle results under tests/golden belong to the graphs the
seeded generators produce today (same CSR hash), and satisfy the census
invariants (class counts sum to C(n, k); the 3- and 4-vertex non-induced
counts agree with the stored sums)."""
import json
import os
from math import comb

import pytest

import graphgen as gg
from gpu_util import graph_hash

HERE = os.path.join(os.path.dirname(__file__), "golden")
MAKERS = {"chung_lu": lambda: gg.config_chung_lu(1), "er500": lambda: gg.config_er500(0), "two_hubs": lambda: gg.two_hubs()}


@pytest.mark.parametrize("name", sorted(MAKERS))
def test_golden_matches_generator_and_invariants(name):
    path = os.path.join(HERE, f"census_{name}.json")
    with open(path) as f:
        gold = json.load(f)
    g = MAKERS[name]()
    assert gold["sha256"] == graph_hash(g), "generator output drifted from the stored oracle result"
    assert (gold["n"], gold["m"]) == (g.n, g.m)
    n = g.n
    for k, key in ((3, "c3"), (4, "c4"), (5, "c5")):
        vals = [int(x) for x in gold[key]]
        assert min(vals) >= 0 and sum(vals) == comb(n, k), key
    n4 = [int(x) for x in gold["n4"]]
    sums = {k: int(v) for k, v in gold["sums"].items()}
    # non-induced 4-cycles, diamonds, 4-cliques; wedges and triangles
    assert (n4[3], n4[4], n4[5]) == (sums["C4"], sums["D"], sums["K4"])
    assert (int(gold["n3"][2]), int(gold["n3"][3])) == (sums["W"], sums["T"])
