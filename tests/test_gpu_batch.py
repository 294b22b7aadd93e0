"""Batched census (one fused pass over the block-diagonal union with per-graph
accumulators): every member's result equals its single-graph census, and the
oracle's, bit for bit."""
import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_util import assert_same_census, gpu_census

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1610_09411_gb300 import build
    build.build()


def _pack(graphs):
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    rps, cols, base = [], [], 0
    for k, g in enumerate(graphs):
        voff[k + 1] = voff[k] + g.n
        rps.append(g.row_ptr[:-1] + base)
        cols.append(g.col)
        base += g.nnz
    rp = np.concatenate(rps + [np.array([base])]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    return voff, rp, col


def test_batch_mixed_members_match_oracle():
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.empty(0), gg.complete(7), gg.empty(3), gg.star(40), gg.cycle(5), gg.path(4),
              gg.erdos_renyi(60, 0.2, 3), gg.barabasi_albert(80, 3, 4), gg.complete_bipartite(2, 30),
              gg.chung_lu(300, 2.1, 6, 60, 5), gg.empty(6), gg.petersen(), gg.complete(70)]
    res = esc.escape_census5_batch(*_pack(graphs))
    assert len(res) == len(graphs)
    for g, r in zip(graphs, res):
        assert_same_census(r, oracle.census(g))


@pytest.mark.parametrize("mode", ["3", "1"])
def test_batch_in_every_pair_mode_matches_oracle(mode, monkeypatch):
    """A batch with every pair item taken as heavy, counted in windows of 64
    ranks (mode 3) or with tagged global counters only (mode 1), instead of
    the single window batches use by default."""
    from paper_1610_09411_gb300 import escape as esc
    monkeypatch.setenv("ESC_PAIR_WINDOW", mode)
    monkeypatch.setenv("ESC_PAIR_WIN_WORDS", "32")
    monkeypatch.setenv("ESC_PAIR_SMALL_W", "1")
    monkeypatch.setenv("ESC_PAIR_LARGE_W", "1")
    graphs = [gg.complete(9), gg.erdos_renyi(60, 0.3, 4), gg.empty(2), gg.barabasi_albert(120, 4, 2),
              gg.chung_lu(400, 2.1, 8, 80, 6), gg.petersen()]
    res = esc.escape_census5_batch(*_pack(graphs))
    for g, r in zip(graphs, res):
        assert_same_census(r, oracle.census(g))


def test_batch_workload_sample_matches_single_calls():
    from paper_1610_09411_gb300 import escape as esc
    graphs = gg.batch_graphs(24, 17, n_lo=20, n_hi=400)
    res = esc.escape_census5_batch(*_pack(graphs))
    for g, r in zip(graphs, res):
        assert_same_census(r, gpu_census(g))


def test_batch_device_pointers():
    import torch
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.erdos_renyi(50, 0.3, s) for s in range(5)]
    voff, rp, col = _pack(graphs)
    res = esc.escape_census5_batch(torch.from_numpy(voff).cuda(), torch.from_numpy(rp).cuda(),
                                   torch.from_numpy(col).cuda())
    for g, r in zip(graphs, res):
        assert_same_census(r, oracle.census(g))


def test_batch_rejects_id_outside_its_graph():
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.complete(4), gg.complete(4)]
    voff, rp, col = _pack(graphs)
    col = col.copy()
    col[0] = 5                       # graph 0 has 4 vertices
    with pytest.raises(esc.EscapeError) as ei:
        esc.escape_census5_batch(voff, rp, col)
    assert ei.value.code == 1


def test_batch_normalize_flag():
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.erdos_renyi(40, 0.2, 1), gg.barabasi_albert(30, 2, 2)]
    voff, rp, col = _pack(graphs)
    # duplicate every entry of graph 1's first row and add a self-loop in graph 0
    res = esc.escape_census5_batch(voff, rp, col, flags=esc.ESCAPE_NORMALIZE)
    for g, r in zip(graphs, res):
        assert_same_census(r, oracle.census(g))


def test_batch_in_chunks_matches_one_chunk(monkeypatch):
    """A batch counted in several chunks (a small work-space budget forces
    them) gives every graph's census, the same as one chunk and the oracle."""
    from gpu_util import gpu_batch
    graphs = [gg.batch_member(k, 2024, n_hi=300) for k in range(18)] + [gg.complete(30), gg.empty(2)]
    one = gpu_batch(graphs)
    monkeypatch.setenv("ESC_BATCH_CHUNK_MB", "4")
    many = gpu_batch(graphs, device=True)
    for g, a, b in zip(graphs, one, many):
        assert_same_census(b, a)
    for g, b in list(zip(graphs, many))[::5]:
        assert_same_census(b, oracle.census(g))
