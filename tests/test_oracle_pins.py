"""Pins for the CPU oracle: checks against things other than the oracle itself.

* the paper's printed 21x21 matrices A and A^-1 (App. B; golden fixtures);
* brute force over every 5-subset (the definition of the induced census);
* closed forms (K_n, stars, cycles, K_{2,b}, the Petersen graph);
* invariants (class sums = C(n,k), per-element identities, relabelling,
  complement duality).
A plausible slip in any closed form, sign, index or operand changes at least
one of these (see test_planted_mistakes_are_caught).
"""
import os
from math import comb

import numpy as np
import pytest

import graphgen as gg
import oracle

GOLDEN = os.path.join(os.path.dirname(__file__), "golden")


def _read_matrix(name):
    rows = []
    with open(os.path.join(GOLDEN, name)) as f:
        for line in f:
            if line.strip() and not line.startswith("#"):
                rows.append([int(x) for x in line.split()])
    return rows


# ----------------------------------------------------------------- matrices (App. B)

def test_matrix_matches_printed_21x21():
    A = oracle.matrix(5)
    printed = _read_matrix("paper_matrix_A.txt")
    assert len(printed) == 21
    assert [row[:21] for row in A[:21]] == printed


def test_inverse_matches_printed_and_sign_rule():
    A = oracle.matrix(5)
    Ainv = _read_matrix("paper_matrix_Ainv.txt")
    # A . A^-1 = I on the 21 connected classes (printed inverse)
    for i in range(21):
        for j in range(21):
            s = sum(A[i][k] * Ainv[k][j] for k in range(21))
            assert s == (1 if i == j else 0)
    # A^-1_ij = (-1)^(e_j - e_i) A_ij, e = edge count (sum of a column of A = 2^e)
    e = [(sum(A[i][j] for i in range(34))).bit_length() - 1 for j in range(34)]
    for i in range(21):
        for j in range(21):
            assert Ainv[i][j] == (-1) ** (e[j] - e[i]) * A[i][j]


def test_catalogue_is_complete():
    # every 10-bit 5-vertex graph falls in one of 34 classes, each class non-empty;
    # class sizes (labelled graphs per class) sum to 2^10
    seen = {}
    for mask in range(1 << 10):
        c = oracle.classify(5, mask)
        assert 0 <= c < 34
        seen[c] = seen.get(c, 0) + 1
    assert len(seen) == 34 and sum(seen.values()) == 1024
    assert len({oracle.classify(4, m) for m in range(64)}) == 11
    assert len({oracle.classify(3, m) for m in range(8)}) == 4
    # 21 connected classes have >= 4 edges and are connected; class 8 is the 5-cycle
    A = oracle.matrix(5)
    e = [(sum(A[i][j] for i in range(34))).bit_length() - 1 for j in range(34)]
    assert e[7] == 5 and e[20] == 10 and e[21] == 0


# ----------------------------------------------------------------- brute force

def _graphs_small():
    out = [gg.complete(5), gg.complete(7), gg.petersen(), gg.star(8), gg.cycle(7),
           gg.complete_bipartite(2, 5), gg.complete_bipartite(3, 4), gg.empty(6), gg.path(9),
           gg.disjoint_union([gg.complete(4), gg.cycle(5), gg.star(4)])]
    for s in range(8):
        out.append(gg.erdos_renyi(10 + s, [0.2, 0.35, 0.5, 0.7, 0.9][s % 5], 100 + s))
    for s in range(4):
        out.append(gg.barabasi_albert(15 + s, 2 + s % 3, 200 + s))
    out.append(gg.chung_lu(40, 2.1, 5, 20, 9))
    out.append(gg.rmat(5, 4, 0.57, 0.19, 0.19, 4))
    return out


@pytest.mark.parametrize("g", _graphs_small(), ids=lambda g: g.name)
def test_census_equals_brute_force(g):
    b = oracle.brute_census(g)
    c = oracle.census(g)
    assert c["c3"] == b["c3"]
    assert c["c4"] == b["c4"]
    assert c["c5"] == b["c5"]


def test_census_equals_brute_force_n25_and_n40():
    for g in (gg.erdos_renyi(25, 0.3, 5), gg.barabasi_albert(25, 3, 6), gg.erdos_renyi(40, 0.15, 8)):
        assert oracle.census(g)["c5"] == oracle.brute_census(g)["c5"]


def test_non_induced_is_A_times_induced():
    g = gg.erdos_renyi(14, 0.45, 31)
    c = oracle.census(g)
    A = oracle.matrix(5)
    assert c["n5"] == [sum(A[i][j] * c["c5"][j] for j in range(34)) for i in range(34)]


# ----------------------------------------------------------------- closed forms

@pytest.mark.parametrize("n", [5, 6, 9, 13, 24])
def test_complete_graph(n):
    c = oracle.census(gg.complete(n))["c5"]
    assert c[20] == comb(n, 5) and sum(c) == comb(n, 5)


@pytest.mark.parametrize("n", [5, 8, 30, 101])
def test_star(n):
    c = oracle.census(gg.star(n))["c5"]
    assert c[0] == comb(n - 1, 4) and c[21] == comb(n - 1, 5)
    assert sum(c) == c[0] + c[21]


@pytest.mark.parametrize("n", [6, 7, 11, 50])
def test_cycle_paths(n):
    c = oracle.census(gg.cycle(n))["c5"]
    assert c[2] == n            # induced P5: the n runs of 5 consecutive vertices


def test_five_cycle_graph():
    c = oracle.census(gg.cycle(5))["c5"]
    assert c[7] == 1 and sum(c) == 1


@pytest.mark.parametrize("b", [3, 4, 10, 40])
def test_k2b(b):
    c = oracle.census(gg.complete_bipartite(2, b))["c5"]
    assert c[12] == comb(b, 3) and c[0] == 2 * comb(b, 4) and c[21] == comb(b, 5)
    assert sum(c) == c[12] + c[0] + c[21]


def test_petersen_twelve_five_cycles():
    c = oracle.census(gg.petersen())
    assert c["c5"][7] == 12 and c["n5"][7] == 12     # girth 5: every 5-cycle is induced


def test_worked_example_pattern2():
    """Sec. 5 derives N2 = sum over ordered edges (d_j - 1) C(d_i - 1, 2) - 2 TT."""
    g = gg.erdos_renyi(15, 0.4, 77)
    S = oracle.raw_sums(g)
    d = g.degrees()
    s = 0
    for u in range(g.n):
        for v in g.col[g.row_ptr[u]:g.row_ptr[u + 1]]:
            s += (int(d[v]) - 1) * comb(int(d[u]) - 1, 2)
    assert oracle.noninduced_from_sums(S)["n5"][1] == s - 2 * S["TT"]
    assert oracle.census(g)["n5"][1] == sum(oracle.matrix(5)[1][j] * x
                                            for j, x in enumerate(oracle.brute_census(g)["c5"]))


# ----------------------------------------------------------------- invariants

@pytest.mark.parametrize("seed", range(3))
def test_class_sums_and_nonnegative(seed):
    g = gg.chung_lu(300, 2.1, 6, 60, seed)
    c = oracle.census(g)
    n = g.n
    assert sum(c["c5"]) == comb(n, 5) and sum(c["c4"]) == comb(n, 4) and sum(c["c3"]) == comb(n, 3)
    assert min(c["c5"] + c["c4"] + c["c3"]) >= 0


def test_per_element_identities():
    g = gg.barabasi_albert(200, 4, 3)
    c = oracle.census(g, per_element=True)
    S, pe = c["sums"], c["per_element"]
    assert int(pe["T_e"].sum()) == 2 * 3 * S["T"]       # both slots of every edge
    assert int(pe["t_i"].sum()) == 3 * S["T"]
    assert int(pe["C4_e"].sum()) == 2 * 4 * S["C4"]
    assert int(pe["C4_i"].sum()) == 4 * S["C4"]
    assert int(pe["K4_e"].sum()) == 2 * 6 * S["K4"]
    assert int(pe["K4_i"].sum()) == 4 * S["K4"]
    # T(e) = |N(u) cap N(v)| straight from the adjacency matrix
    M = np.zeros((g.n, g.n), dtype=np.int64)
    s, d = g.edges()
    M[s, d] = M[d, s] = 1
    M2 = M @ M
    src = np.repeat(np.arange(g.n), g.degrees())
    assert np.array_equal(pe["T_e"].astype(np.int64), M2[src, g.col])
    assert np.array_equal(pe["t_i"].astype(np.int64), np.diag(M2 @ M) // 2)
    # 4-cycles through a vertex / an edge, from pair counts W = M^2 (j != i)
    d = M.sum(1)
    W = M2.copy()
    np.fill_diagonal(W, 0)
    assert np.array_equal(pe["C4_i"].astype(np.int64), (W * (W - 1) // 2).sum(1))
    C4e = (W - 1) @ M                       # sum_j M[k,j] (W[i,j] - 1) over all j ...
    C4e = C4e + M                           # ... the j = i term is W[i,i]-1 = -1: add it back
    assert np.array_equal(pe["C4_e"].astype(np.int64), C4e[src, g.col])
    # 4-cliques through an edge: edges inside the common neighbourhood
    k4 = np.array([(M[u] * M[v]) @ M @ (M[u] * M[v]) // 2 for u, v in zip(src, g.col)])
    assert np.array_equal(pe["K4_e"].astype(np.int64), k4)


def test_relabel_invariance():
    g = gg.chung_lu(400, 2.1, 8, 100, 4)
    perm = np.random.default_rng(5).permutation(g.n)
    a = oracle.census(g)
    b = oracle.census(gg.relabel(g, perm))
    assert a["c5"] == b["c5"] and a["c4"] == b["c4"]


def _complement_map(k):
    full = (1 << (k * (k - 1) // 2)) - 1
    ncls = oracle.NCLS[k]
    mp = {}
    for mask in range(full + 1):
        mp[oracle.classify(k, mask)] = oracle.classify(k, full ^ mask)
    assert len(mp) == ncls
    return mp


@pytest.mark.parametrize("g", [gg.erdos_renyi(60, 0.1, 3), gg.barabasi_albert(70, 2, 4)],
                         ids=lambda g: g.name)
def test_complement_duality(g):
    a = oracle.census(g)
    b = oracle.census(gg.complement(g))
    for k, key in ((4, "c4"), (5, "c5")):
        mp = _complement_map(k)
        assert all(b[key][mp[c]] == a[key][c] for c in range(oracle.NCLS[k]))


# ----------------------------------------------------------------- planted mistakes

def test_planted_mistakes_are_caught():
    """Forms of the closed formulas as the paper prints them (or with one slip)
    must disagree with brute force, so the pins above would catch them."""
    g = gg.erdos_renyi(13, 0.6, 12)
    truth = oracle.brute_census(g)["c5"]
    S = oracle.raw_sums(g)
    mutations = {
        "N4 printed as TT": lambda S: S.__setitem__("N4", S["TT"]),
        "N18 without the 1/2": lambda S: S.__setitem__("N18X4", 2 * S["N18X4"]),
        "N20 with -4 K4": lambda S: S.__setitem__("N20", S["N20"] - 4 * S["K4"]),
        "N16 without -12 K4": lambda S: S.__setitem__("N16A", S["N16A"] + 12 * S["K4"]),
        "N10 with (d_k - 1) and -4 K4": lambda S: S.__setitem__("N10A", S["N10A"] + 2 * S["D"] + 8 * S["K4"]),
        "5-cycle without Z": lambda S: S.__setitem__("N8Z", 0),
        "N5 sign slip": lambda S: S.__setitem__("N5A", S["N5A"] + 8 * S["D"]),
        "N13 off by one pair": lambda S: S.__setitem__("N13", S["N13"] + 1),
    }
    for name, mut in mutations.items():
        T = dict(S)
        mut(T)
        c = oracle.induced_from_noninduced(oracle.noninduced_from_sums(T))["c5"]
        assert c != truth, name


def test_single_element_definitions_match_full_census():
    """The sampled-check helpers (single edges / vertices from their
    definitions) agree with the whole-graph per-element arrays."""
    g = gg.chung_lu(600, 2.1, 8, 80, 6)
    pe = oracle.census(g, per_element=True)["per_element"]
    src = np.repeat(np.arange(g.n), g.degrees())
    idx = np.arange(0, g.nnz, 5)
    e = oracle.edge_elements(g, src[idx], g.col[idx])
    for k in ("T_e", "K4_e", "C4_e"):
        assert np.array_equal(e[k], pe[k][idx]), k
    vs = np.arange(0, g.n, 4)
    v = oracle.vertex_elements(g, vs)
    for k in ("t_i", "C4_i"):
        assert np.array_equal(v[k], pe[k][vs]), k


# ----------------------------------------------------------------- OpenMP build

def test_parallel_build_equals_brute_force_and_serial():
    """The OpenMP build of the same oracle source (used to write the stored
    results of the large workloads) gives brute force's counts and the serial
    build's sums and per-element arrays on every brute-force graph."""
    for g in _graphs_small() + [gg.erdos_renyi(40, 0.15, 8), gg.chung_lu(3000, 2.1, 8, 300, 5)]:
        par = oracle.census(g, per_element=True, parallel=True)
        ser = oracle.census(g, per_element=True)
        assert par["sums"] == ser["sums"], g.name
        for k in ser["per_element"]:
            assert np.array_equal(par["per_element"][k], ser["per_element"][k]), (g.name, k)
        if g.n <= 40:
            assert par["c5"] == oracle.brute_census(g)["c5"], g.name


def test_wedge_diamond_sums_equal_the_census_sums():
    """W, T and D alone (the unit counts of the byte model for the largest
    workload) agree with the full census's sums and with brute force."""
    for g in _graphs_small() + [gg.chung_lu(3000, 2.1, 8, 300, 5)]:
        s = oracle.census(g)["sums"]
        for par in (False, True):
            w = oracle.wedge_diamond_sums(g, parallel=par)
            assert w == {"W": s["W"], "T": s["T"], "D": s["D"]}, g.name
        if g.n <= 40:
            b = oracle.brute_census(g)
            # 3-vertex wedges (induced) + 3 x triangles = W; 4-vertex induced diamonds + 6 x K4 = D
            assert w["W"] == b["c3"][2] + 3 * b["c3"][3]
            assert w["T"] == b["c3"][3]
            assert w["D"] == b["c4"][4] + 6 * b["c4"][5]
        # the same sums are the census's non-induced wedges, triangles and diamonds
        c = oracle.census(g)
        assert (c["n3"][2], c["n3"][3], c["n4"][4]) == (w["W"], w["T"], w["D"]), g.name


def test_pair_sums_equal_the_census_and_closed_forms():
    """C4 and N13 (non-induced K2,3, class 13 of the connected patterns) from
    the two-hop pair counts alone agree with the census (serial and OpenMP
    builds) and with the closed forms of K_n and K_{2,b}."""
    for g in _graphs_small() + [gg.chung_lu(3000, 2.1, 8, 300, 5), gg.config_rmat(11, 2)]:
        c = oracle.census(g)
        for par in (False, True):
            assert oracle.pair_sums(g, parallel=par) == {"C4": c["n4"][3], "N13": c["n5"][12]}, g.name
    for n in (4, 5, 9, 17):
        assert oracle.pair_sums(gg.complete(n)) == {"C4": 3 * comb(n, 4), "N13": comb(n, 2) * comb(n - 2, 3)}
    for b in (1, 2, 3, 7, 30):
        assert oracle.pair_sums(gg.complete_bipartite(2, b)) == {"C4": comb(b, 2), "N13": comb(b, 3)}


def test_clique4_count_equals_the_census_and_closed_forms():
    """The 4-cliques counted alone (each at its lowest vertex, as a triangle
    of G[N+(x)]) agree with the census (serial and OpenMP builds), with
    C(n,4) on K_n and with zero on triangle-free graphs."""
    for g in _graphs_small() + [gg.chung_lu(3000, 2.1, 8, 300, 5), gg.config_rmat(11, 2)]:
        k4 = oracle.census(g)["n4"][5]
        for par in (False, True):
            assert oracle.clique4_count(g, parallel=par) == k4, g.name
    for n in (3, 4, 5, 12, 30):
        assert oracle.clique4_count(gg.complete(n)) == comb(n, 4)
    for g in (gg.complete_bipartite(7, 9), gg.petersen(), gg.cycle(12)):
        assert oracle.clique4_count(g) == 0


def test_clique5_count_equals_the_census_and_closed_forms():
    """The 5-cliques counted alone (each at its lowest vertex, as a 4-clique
    of G[N+(x)] with bit sets) agree with the census's bipyramid count
    (serial and OpenMP builds), with C(n,5) on K_n, with zero on graphs without
    K5, and with brute force on small random graphs."""
    for g in _graphs_small() + [gg.chung_lu(3000, 2.1, 8, 300, 5), gg.config_rmat(11, 2),
                                gg.erdos_renyi(120, 0.5, 3)]:
        k5 = oracle.census(g)["n5"][20]
        for par in (False, True):
            assert oracle.clique5_count(g, parallel=par) == k5, g.name
        if g.n <= 40:
            assert k5 == oracle.brute_census(g)["c5"][20] or g.n < 5
    for n in (4, 5, 6, 13, 64, 65, 70, 130):
        assert oracle.clique5_count(gg.complete(n)) == comb(n, 5)
    for g in (gg.complete_bipartite(7, 9), gg.petersen(), gg.complete(4)):
        assert oracle.clique5_count(g) == 0
