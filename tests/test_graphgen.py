"""Seeded input generators: determinism and CSR invariants (no census arithmetic)."""
import numpy as np
import pytest

import graphgen as gg


def _check_csr(g):
    assert g.row_ptr[0] == 0 and len(g.row_ptr) == g.n + 1
    assert np.all(np.diff(g.row_ptr) >= 0)
    src = np.repeat(np.arange(g.n), g.degrees())
    assert np.all(g.col >= 0) and np.all(g.col < g.n)
    assert not np.any(src == g.col)                     # no self-loops
    for u in range(min(g.n, 200)):
        row = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        assert np.all(np.diff(row) > 0)                 # sorted, no duplicates
    key = src.astype(np.int64) * g.n + g.col
    rkey = g.col.astype(np.int64) * g.n + src
    assert np.array_equal(np.sort(key), np.sort(rkey))  # symmetric


@pytest.mark.parametrize("make", [
    lambda: gg.erdos_renyi(300, 0.02, 7),
    lambda: gg.barabasi_albert(400, 3, 5),
    lambda: gg.chung_lu(2000, 2.1, 8, 200, 3),
    lambda: gg.rmat(10, 8, 0.57, 0.19, 0.19, 2),
])
def test_generators_valid_and_deterministic(make):
    g1, g2 = make(), make()
    _check_csr(g1)
    assert np.array_equal(g1.row_ptr, g2.row_ptr) and np.array_equal(g1.col, g2.col)


def test_er500_size():
    g = gg.config_er500(0)
    assert g.n == 500
    assert 1200 < g.m < 1800        # p * C(500, 2) = 1497


def test_seed_changes_graph():
    a, b = gg.erdos_renyi(100, 0.1, 1), gg.erdos_renyi(100, 0.1, 2)
    assert not (a.m == b.m and np.array_equal(a.col, b.col))


def test_structured_graphs():
    assert gg.complete(6).m == 15
    assert gg.star(7).m == 6
    assert gg.cycle(8).m == 8
    assert gg.complete_bipartite(2, 5).m == 10
    assert gg.petersen().m == 15 and np.all(gg.petersen().degrees() == 3)
    assert gg.complement(gg.complete(5)).m == 0
    g = gg.from_edges(5, [0, 1, 1, 3, 3], [1, 0, 1, 4, 4])   # duplicates, loop, both directions
    assert g.m == 2


def test_batch_graphs_mix():
    gs = gg.batch_graphs(6, 11)
    assert len(gs) == 6
    for g in gs:
        assert 20 <= g.n <= 2000
        _check_csr(g)
