"""GPU parity: the CUDA census through the C ABI against the CPU oracle.

Bar: bit-exact (all counts are integers).  Cases span several CTAs/tiles,
ragged tails (out-degrees across the 32-lane and 64-bit word boundaries of the
kernels), hub-heavy graphs, empty and tiny graphs, the ER(500) workload for
ten seeds, the Chung-Lu workload (stored oracle result) and the R-MAT scale-22
workload at full size (sampled per-element values and invariants).
"""
import json
import os
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle
from gpu_util import assert_same_census, gpu_batch, gpu_census, graph_hash

pytestmark = pytest.mark.gpu

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1610_09411_gb300 import build
    build.build()


# ------------------------------------------------------------------ small / structured

def _structured():
    return [gg.empty(0), gg.empty(1), gg.empty(4), gg.empty(9), gg.path(2), gg.path(4), gg.complete(4),
            gg.complete(5), gg.complete(12), gg.star(6), gg.star(300), gg.cycle(5), gg.cycle(40),
            gg.petersen(), gg.complete_bipartite(2, 3), gg.complete_bipartite(2, 70),
            gg.complete_bipartite(5, 40),
            gg.disjoint_union([gg.complete(6), gg.cycle(7), gg.star(9), gg.empty(3)])]


@pytest.mark.parametrize("g", _structured(), ids=lambda g: f"{g.name}_n{g.n}")
def test_structured_graphs_match_oracle(g):
    assert_same_census(gpu_census(g), oracle.census(g))


@pytest.mark.parametrize("seed", range(6))
def test_small_random_match_brute_force(seed):
    g = [gg.erdos_renyi(14, 0.5, seed), gg.barabasi_albert(18, 3, seed), gg.chung_lu(24, 2.1, 6, 20, seed)][seed % 3]
    got = gpu_census(g)
    b = oracle.brute_census(g)
    assert got["c5"] == b["c5"] and got["c4"] == b["c4"] and got["c3"] == b["c3"]


@pytest.mark.parametrize("make", [
    lambda: gg.complete(33),            # out-degrees 0..32: the 32-lane boundary
    lambda: gg.complete(66),            # bit rows spanning two 64-bit words
    lambda: gg.complete(131),           # three words, many 5-cliques
    lambda: gg.erdos_renyi(400, 0.35, 1),
    lambda: gg.erdos_renyi(3000, 0.01, 2),
    lambda: gg.barabasi_albert(5000, 6, 3),
    lambda: gg.chung_lu(20000, 2.1, 10, 2000, 4),
    lambda: gg.rmat(12, 16, 0.57, 0.19, 0.19, 5),
    lambda: gg.disjoint_union([gg.star(2000), gg.complete_bipartite(3, 500), gg.complete(40)]),
], ids=["K33", "K66", "K131", "er400_dense", "er3000", "ba5000", "cl20000", "rmat12", "hubs"])
def test_ragged_and_hub_graphs_match_oracle(make):
    g = make()
    assert_same_census(gpu_census(g), oracle.census(g))


# ------------------------------------------------------------------ per-element arrays (Thm 7)

@pytest.mark.parametrize("make", [lambda: gg.config_er500(3), lambda: gg.barabasi_albert(3000, 5, 1),
                                  lambda: gg.chung_lu(20000, 2.1, 10, 2000, 4), lambda: gg.complete(70)],
                         ids=["er500", "ba3000", "cl20000", "K70"])
def test_per_element_arrays_match_oracle(make):
    g = make()
    got = gpu_census(g, per_element=True)["per_element"]
    want = oracle.census(g, per_element=True)["per_element"]
    for k in ("T_e", "t_i", "C4_e", "C4_i", "K4_e", "K4_i"):
        assert np.array_equal(got[k], want[k]), k


# ------------------------------------------------------------------ workloads

@pytest.mark.parametrize("seed", range(10))
def test_er500_workload(seed):
    g = gg.config_er500(seed)
    assert_same_census(gpu_census(g), oracle.census(g))


def _golden(name):
    path = os.path.join(GOLDEN, f"census_{name}.json")
    if not os.path.exists(path):
        return None
    with open(path) as f:
        return json.load(f)


def test_chung_lu_workload():
    """Chung-Lu n=262144, exponent 2.1, mean 16, clip 8192 (~2M edges)."""
    from gpu_util import graph_hash
    g = gg.config_chung_lu(1)
    got = gpu_census(g, device=True)
    gold = _golden("chung_lu")
    if gold is not None and gold["sha256"] == graph_hash(g):
        want = {k: [int(x) for x in gold[k]] for k in ("c3", "c4", "c5", "n3", "n4", "n5")}
    else:   # the regenerated graph differs from the stored one: compute live
        want = oracle.census(g)
    assert_same_census(got, want)


def test_two_hubs_wide_counts():
    """Two hubs of degree > 2^16 with > 2^16 common neighbours: the pair and
    5-cycle counts at the hubs leave 16 bits (stored oracle result)."""
    from gpu_util import graph_hash
    g = gg.two_hubs()
    got = gpu_census(g, device=True)
    gold = _golden("two_hubs")
    if gold is not None and gold["sha256"] == graph_hash(g):
        want = {k: [int(x) for x in gold[k]] for k in ("c3", "c4", "c5", "n3", "n4", "n5")}
    else:
        want = oracle.census(g)
    assert_same_census(got, want)


@pytest.mark.parametrize("win_words,make", [
    (1, lambda: gg.petersen()),
    (1, lambda: gg.complete(30)),
    (3, lambda: gg.disjoint_union([gg.star(40), gg.complete(12), gg.cycle(7)])),
    (2, lambda: gg.erdos_renyi(60, 0.3, 5)),
    (64, lambda: gg.barabasi_albert(2000, 4, 6)),
    (64, lambda: gg.chung_lu(5000, 2.1, 10, 1000, 3)),
    (200, lambda: gg.config_rmat(12, 3)),
    (4096, lambda: gg.chung_lu(20000, 2.1, 10, 2000, 8)),
], ids=["petersen-w1", "K30-w1", "union-w3", "er60-w2", "ba2000-w64", "cl5000-w64", "rmat12-w200", "cl20000-w4096"])
def test_pair_sweep_in_many_windows_matches_oracle(win_words, make, monkeypatch):
    """Every pair-sweep item taken as heavy and counted in windows of
    2 x win_words ranks (many windows per item: cursors, the dense 16-bit
    array, the top window on chip); the census equals the oracle's."""
    monkeypatch.setenv("ESC_PAIR_SMALL_W", "1")
    monkeypatch.setenv("ESC_PAIR_LARGE_W", "1")
    monkeypatch.setenv("ESC_PAIR_WIN_WORDS", str(win_words))
    g = make()
    assert_same_census(gpu_census(g), oracle.census(g))


@pytest.mark.parametrize("mode", ["3", "2", "1"])
def test_two_hubs_in_every_pair_mode(mode, monkeypatch):
    """Counts above 2^16 at two hubs (the 64-bit counters of ranks >= jbig)
    with the windowed heavy items in windows of 8192 ranks, the single window
    and no window: the stored oracle result."""
    monkeypatch.setenv("ESC_PAIR_WINDOW", mode)
    monkeypatch.setenv("ESC_PAIR_WIN_WORDS", "4096")
    g = gg.two_hubs()
    gold = _golden("two_hubs")
    assert gold is not None and gold["sha256"] == graph_hash(g)
    got = gpu_census(g, device=True)
    assert_same_census(got, {k: [int(x) for x in gold[k]] for k in ("c3", "c4", "c5", "n3", "n4", "n5")})


@pytest.mark.parametrize("make", [lambda: gg.config_er500(1), lambda: gg.complete(40),
                                  lambda: gg.chung_lu(20000, 2.1, 10, 2000, 4), lambda: gg.barabasi_albert(3000, 5, 2),
                                  lambda: gg.disjoint_union([gg.star(3000), gg.complete(70), gg.empty(4)]),
                                  lambda: gg.empty(3)],
                         ids=["er500", "K40", "cl20000", "ba3000", "star_union", "empty3"])
def test_census4_alone(make):
    """escape_census4 (the 3- and 4-vertex census without the 5-vertex
    sweeps) gives the oracle's counts, the same as the 3- and 4-vertex part of
    escape_census5, and the same per-element arrays."""
    from paper_1610_09411_gb300 import escape as esc
    g = make()
    h = esc.escape_load_csr(g.n, g.row_ptr, g.col)
    try:
        esc.escape_set_options(h, True)
        r4 = esc.escape_census4(h)
        pe4 = esc.escape_per_element(h) if g.m > 0 else None
        r5 = esc.escape_census5(h)
        pe5 = esc.escape_per_element(h) if g.m > 0 else None
    finally:
        esc.escape_free(h)
    keys = ("c3", "c4", "n3", "n4")
    assert_same_census(r4, r5, keys)
    assert_same_census(r4, oracle.census(g), keys)
    if pe4 is not None:
        for k in pe4:
            assert np.array_equal(pe4[k], pe5[k]), k


def test_censuses_on_concurrent_host_threads():
    """Censuses issued at the same time from several host threads, each on its
    own stream, over graphs whose kernels need different shared-memory sizes
    (as a serving loop with several workers does), give each graph's result
    alone."""
    import threading
    import torch
    from paper_1610_09411_gb300 import escape as esc
    graphs = [gg.complete(40), gg.complete(90), gg.chung_lu(6000, 2.1, 10, 1500, 3),
              gg.barabasi_albert(4000, 6, 2), gg.disjoint_union([gg.star(3000), gg.complete(70)])]
    want = [gpu_census(g) for g in graphs]
    errors, got = [], {}

    def worker(k):
        try:
            st = torch.cuda.Stream()
            for rnd in range(3):
                for t, g in enumerate(graphs):
                    if (t + k + rnd) % 2:
                        continue
                    h = esc.escape_load_csr(g.n, g.row_ptr, g.col, stream=st.cuda_stream)
                    try:
                        got[(k, rnd, t)] = esc.escape_census5(h, stream=st.cuda_stream)
                    finally:
                        esc.escape_free(h)
        except Exception as e:      # reported below, on the main thread
            errors.append(e)

    threads = [threading.Thread(target=worker, args=(k,)) for k in range(3)]
    for th in threads:
        th.start()
    for th in threads:
        th.join()
    assert not errors, errors
    assert got
    for (k, rnd, t), r in got.items():
        assert_same_census(r, want[t])


def test_serial_and_concurrent_phases_agree():
    from paper_1610_09411_gb300 import escape as esc
    g = gg.chung_lu(20000, 2.1, 10, 2000, 8)
    h = esc.escape_load_csr(g.n, g.row_ptr, g.col)
    try:
        esc.escape_set_options(h, True, 0, True)
        a = esc.escape_census5(h)
        pa = esc.escape_per_element(h)
        esc.escape_set_options(h, True, 3, False)
        b = esc.escape_census5(h)
        pb = esc.escape_per_element(h)
    finally:
        esc.escape_free(h)
    assert_same_census(a, b)
    for k in pa:
        assert np.array_equal(pa[k], pb[k]), k


def test_device_and_host_pointers_agree():
    g = gg.chung_lu(5000, 2.1, 8, 500, 7)
    assert_same_census(gpu_census(g), gpu_census(g, device=True))


def _check_stored_elements(g, pe, el):
    """Per-element GPU values (input CSR layout) at the stored sample."""
    verts = np.array(el["vertices"], dtype=np.int64)
    for k in ("t_i", "C4_i", "K4_i"):
        if k in el:
            assert [int(x) for x in pe[k][verts]] == [int(x) for x in el[k]], k
    slots = []
    for u, v in el["edges"]:
        row = g.col[g.row_ptr[u]:g.row_ptr[u + 1]]
        q = int(np.searchsorted(row, v))
        assert row[q] == v
        slots.append(int(g.row_ptr[u]) + q)
    slots = np.array(slots, dtype=np.int64)
    for k in ("T_e", "C4_e", "K4_e"):
        if k in el:
            assert [int(x) for x in pe[k][slots]] == [int(x) for x in el[k]], k


def test_rmat_scale20_full_census_matches_stored_oracle():
    """R-MAT scale 20 (the headline generator and parameters at a quarter of
    the size; stored oracle result of the whole census): every induced and
    non-induced count bit for bit, and the per-element values at the sampled
    vertices and edges (the highest-degree ones among them) when stored."""
    path = os.path.join(GOLDEN, "census_rmat20.json")
    if not os.path.exists(path):
        pytest.skip("no stored oracle result")
    with open(path) as f:
        gold = json.load(f)
    g = gg.config_rmat(20, 1)
    assert gold["sha256"] == graph_hash(g)
    got = gpu_census(g, per_element="elements" in gold, device=True)
    for key in ("c3", "c4", "c5", "n3", "n4", "n5"):
        assert got[key] == [int(x) for x in gold[key]], key
    if "elements" in gold:
        _check_stored_elements(g, got["per_element"], gold["elements"])


def test_rmat_scale22_full_size():
    """R-MAT scale 22 (the benchmark workload): the full census against the
    stored oracle result when one exists; otherwise the invariants of the
    census, and the per-element values at the sampled vertices and edges --
    the ten highest-degree vertices, their mutual edges and first entries among
    them -- against the oracle's single-element definitions (stored, or
    computed here for a sample of non-hub vertices and edges)."""
    g = gg.config_rmat()
    got = gpu_census(g, per_element=True, device=True)
    n = g.n
    path = os.path.join(GOLDEN, "census_rmat22.json")
    if os.path.exists(path):
        with open(path) as f:
            gold = json.load(f)
        assert gold["sha256"] == graph_hash(g)
        for key in ("c3", "c4", "c5", "n3", "n4", "n5"):
            assert got[key] == [int(x) for x in gold[key]], key
    assert sum(got["c5"]) == comb(n, 5) and sum(got["c4"]) == comb(n, 4) and sum(got["c3"]) == comb(n, 3)
    assert min(got["c5"] + got["c4"]) >= 0
    # the oracle's wedges, triangles and diamonds of this graph (stored): the
    # non-induced wedge, triangle and diamond counts
    sums_path = os.path.join(GOLDEN, "sums_rmat22.json")
    if os.path.exists(sums_path):
        with open(sums_path) as f:
            sums = json.load(f)
        assert sums["sha256"] == graph_hash(g)
        assert got["n3"][2] == int(sums["sums"]["W"])
        assert got["n3"][3] == int(sums["sums"]["T"])
        assert got["n4"][4] == int(sums["sums"]["D"])
    # the oracle's pair sums (two-hop counts W(i,j) from every vertex): the
    # 4-cycles and the non-induced K2,3 (class 13 of the connected patterns)
    pairs_path = os.path.join(GOLDEN, "pairs_rmat22.json")
    if os.path.exists(pairs_path):
        with open(pairs_path) as f:
            pairs = json.load(f)
        assert pairs["sha256"] == graph_hash(g)
        assert got["n4"][3] == int(pairs["sums"]["C4"])
        assert got["n5"][12] == int(pairs["sums"]["N13"])
    # the oracle's 4-clique count
    cliques_path = os.path.join(GOLDEN, "cliques_rmat22.json")
    if os.path.exists(cliques_path):
        with open(cliques_path) as f:
            cliques = json.load(f)
        assert cliques["sha256"] == graph_hash(g)
        assert got["n4"][5] == int(cliques["sums"]["K4"])
    # the oracle's 5-clique count (class 21)
    cliques5_path = os.path.join(GOLDEN, "cliques5_rmat22.json")
    if os.path.exists(cliques5_path):
        with open(cliques5_path) as f:
            cliques5 = json.load(f)
        assert cliques5["sha256"] == graph_hash(g)
        assert got["n5"][20] == int(cliques5["sums"]["K5"])
    pe = got["per_element"]
    T = got["n3"][3]
    assert int(pe["T_e"].sum()) == 6 * T and int(pe["t_i"].sum()) == 3 * T
    assert int(pe["C4_e"].sum()) == 8 * got["n4"][3] and int(pe["C4_i"].sum()) == 4 * got["n4"][3]
    assert int(pe["K4_e"].sum()) == 12 * got["n4"][5] and int(pe["K4_i"].sum()) == 4 * got["n4"][5]
    el_path = os.path.join(GOLDEN, "elements_rmat22.json")
    if os.path.exists(el_path):
        with open(el_path) as f:
            el = json.load(f)
        assert el["sha256"] == graph_hash(g)
        _check_stored_elements(g, pe, el["elements"])
    rng = np.random.default_rng(2024)
    src = np.repeat(np.arange(n), g.degrees())
    idx = rng.choice(g.nnz, size=40, replace=False)
    e = oracle.edge_elements(g, src[idx], g.col[idx])
    for k in ("T_e", "K4_e", "C4_e"):
        assert np.array_equal(pe[k][idx], e[k]), k
    deg = g.degrees()
    vs = rng.choice(np.nonzero((deg > 0) & (deg < 20000))[0], size=40, replace=False)
    v = oracle.vertex_elements(g, vs)
    for k in ("t_i", "C4_i"):
        assert np.array_equal(pe[k][vs], v[k]), k


# ------------------------------------------------------------------ input handling

def test_normalize_flag_matches_clean_input():
    from paper_1610_09411_gb300 import escape as esc
    g = gg.erdos_renyi(200, 0.05, 9)
    s, d = g.edges()
    rng = np.random.default_rng(0)
    # messy edge list: both/one direction, duplicates, self-loops, unsorted rows
    us = np.concatenate([s, d[: len(d) // 2], s[:50], np.arange(30)])
    vs = np.concatenate([d, s[: len(s) // 2], d[:50], np.arange(30)])
    order = rng.permutation(len(us))
    us, vs = us[order], vs[order]
    cnt = np.bincount(us, minlength=g.n)
    rp = np.zeros(g.n + 1, dtype=np.int64)
    rp[1:] = np.cumsum(cnt)
    col = vs[np.argsort(us, kind="stable")].astype(np.int32)
    got = esc.census(rp, col, n=g.n, flags=esc.ESCAPE_NORMALIZE)
    assert_same_census(got, oracle.census(g))


@pytest.mark.parametrize("case", ["unsorted", "loop", "asymmetric", "out_of_range", "bad_rowptr"])
def test_invalid_inputs_rejected(case):
    from paper_1610_09411_gb300 import escape as esc
    rp = np.array([0, 2, 4, 6], dtype=np.int64)
    col = np.array([1, 2, 0, 2, 0, 1], dtype=np.int32)       # triangle
    if case == "unsorted":
        col = np.array([2, 1, 0, 2, 0, 1], dtype=np.int32)
    elif case == "loop":
        col = np.array([0, 1, 0, 2, 0, 1], dtype=np.int32)
    elif case == "asymmetric":
        rp = np.array([0, 2, 3, 5], dtype=np.int64)
        col = np.array([1, 2, 0, 0, 1], dtype=np.int32)
    elif case == "out_of_range":
        col = np.array([1, 7, 0, 2, 0, 1], dtype=np.int32)
    elif case == "bad_rowptr":
        rp = np.array([0, 4, 2, 6], dtype=np.int64)
    with pytest.raises(esc.EscapeError) as ei:
        esc.escape_load_csr(3, rp, col)
    assert ei.value.code == 1


@pytest.mark.parametrize("bad", [[0, 4, 2, 6], [0, 9, 4, 6], [0, 2, 9, 6], [0, -2, 4, 6], [0, 2, 4, 5]],
                         ids=["decreasing", "interior_past_nnz", "interior_past_nnz_late", "negative", "end_not_nnz"])
def test_device_row_ptr_checked_on_the_host(bad):
    """Device-memory CSRs: every row offset is copied to the host and checked
    before any kernel indexes col through it, so a malformed row pointer is
    EINVAL for both escape_load_csr and escape_census5_batch."""
    import torch
    from paper_1610_09411_gb300 import escape as esc
    col = torch.tensor([1, 2, 0, 2, 0, 1], dtype=torch.int32, device="cuda")    # a triangle
    rp = torch.tensor(bad, dtype=torch.int64, device="cuda")
    with pytest.raises(esc.EscapeError) as ei:
        esc.escape_load_csr(3, rp, col)
    assert ei.value.code == 1
    if bad[-1] == 6:        # the batch takes its entry count from the last offset
        voff = torch.tensor([0, 3], dtype=torch.int64, device="cuda")
        with pytest.raises(esc.EscapeError) as ei:
            esc.escape_census5_batch(voff, rp, col)
        assert ei.value.code == 1
    # the library is still usable
    good = torch.tensor([0, 2, 4, 6], dtype=torch.int64, device="cuda")
    torch.cuda.synchronize()
    assert esc.census(good, col, n=3)["c3"][3] == 1


def test_batch_matches_single_graph_calls():
    from paper_1610_09411_gb300 import escape as esc
    graphs = gg.batch_graphs(12, 5, n_lo=20, n_hi=300)
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    rps, cols = [], []
    base = 0
    for k, g in enumerate(graphs):
        voff[k + 1] = voff[k] + g.n
        rps.append(g.row_ptr[:-1] + base)
        cols.append(g.col)
        base += g.nnz
    rp = np.concatenate(rps + [np.array([base])]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32)
    res = esc.escape_census5_batch(voff, rp, col)
    for g, r in zip(graphs, res):
        assert_same_census(r, gpu_census(g))
    assert_same_census(res[0], oracle.census(graphs[0]))


# ------------------------------------------------------------------ dense graphs (large out-degrees)

def _closed(n5_idx_vals, n):
    c = [0] * 34
    for i, v in n5_idx_vals:
        c[i] += v
    return c


@pytest.mark.parametrize("n", [1250, 1400])
def test_complete_graph_beyond_the_shared_memory_bit_matrix(n):
    """K_n with out-degrees above what the clique pass's shared-memory bit
    matrix holds: every 5-subset is a 5-clique (class 21), every 4-subset a
    4-clique, every 3-subset a triangle."""
    got = gpu_census(gg.complete(n))
    assert got["c5"] == _closed([(20, comb(n, 5))], n)
    assert got["c4"][5] == comb(n, 4) and sum(got["c4"]) == comb(n, 4)
    assert got["c3"] == [0, 0, 0, comb(n, 3)]


def test_complete_bipartite_beyond_the_shared_memory_bit_matrix():
    """K_{a,b}, a = b = 1300: a 5-subset with k vertices on one side is empty
    (k = 0, 5), a 4-star (k = 1, 4) or K_{2,3} (k = 2, 3)."""
    a = b = 1300
    got = gpu_census(gg.complete_bipartite(a, b))
    want = _closed([(21, comb(a, 5) + comb(b, 5)), (0, a * comb(b, 4) + b * comb(a, 4)),
                    (12, comb(a, 2) * comb(b, 3) + comb(a, 3) * comb(b, 2))], a + b)
    assert got["c5"] == want


def test_dense_batch_member_matches_stored_oracle():
    """Member 24 of the batch workload, G(1250, 0.279) (stored oracle result)."""
    gold_path = os.path.join(GOLDEN, "census_batch24.json")
    if not os.path.exists(gold_path):
        pytest.skip("no stored oracle result")
    with open(gold_path) as f:
        gold = json.load(f)
    g = gg.batch_member(24, 2024)
    assert gold["sha256"] == graph_hash(g)
    got = gpu_census(g)
    for key in ("c3", "c4", "c5", "n3", "n4", "n5"):
        assert got[key] == [int(x) for x in gold[key]], key
    res = gpu_batch([g, gg.batch_member(25, 2024), gg.batch_member(26, 2024)])
    for key in ("c3", "c4", "c5", "n3", "n4", "n5"):
        assert res[0][key] == [int(x) for x in gold[key]], key
