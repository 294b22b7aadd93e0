"""CPU oracle for the ESCAPE 5-vertex census -- TEST INFRASTRUCTURE ONLY.

Only ``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline
leg may import this package.  The CUDA library never calls it; it shares no
code, header or table with it.

Two tiers (see ``escape_oracle.c``):

* ``brute_census``: every 3-, 4- and 5-vertex subset classified by canonical
  form -- the definition of the induced census (Sec. 3.1), small n only.
* ``census``: the paper's method written plainly.  The C part computes the
  per-vertex/per-edge quantities from their definitions and the raw sums; this
  module assembles the non-induced counts N1..N34 from the closed forms in
  exact Python integers and converts them to induced counts with C = A^-1 N
  (App. B), A built by brute force over the pattern catalogue.

Readings of the paper used here (where it is garbled or silent):
  * N3, N4, N5, N10, N16, N18, N20 and the 5-cycle sum are used in their
    corrected forms (the printed forms of Thms 8-11 and 13 fail against brute
    force); every one is pinned by the brute-force tests.
  * Edge sums written with angle brackets (N2, N5, N11) range over both
    orientations of every edge.
  * The 13 disconnected 5-vertex classes include P3+K2 and K3+K2, which the
    paper's figure of disconnected patterns omits.
  * A[i][j] counts spanning subgraphs of class j isomorphic to class i (rows
    are the smaller pattern), which is what the printed matrix holds.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from math import comb

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "escape_oracle.c")
_LIB = os.path.join(_HERE, "liboracle.so")
_LIB_OMP = os.path.join(_HERE, "liboracle_omp.so")
_lock = threading.Lock()
_lib = None
_lib_omp = None

NCLS = {3: 4, 4: 11, 5: 34}

# sum indices, in the order of the enum in escape_oracle.c
SUM_NAMES = [
    "n", "m", "W", "S3", "S4", "T", "EDGE_DD", "TT", "C4", "D", "K4", "N2A", "N3A", "N4",
    "N5A", "N6A", "N7A", "N8M", "N8Z", "N9A", "N10A", "N11", "N12A", "N13", "N14", "N15",
    "N16A", "N17", "N18X4", "N19", "N20", "N21", "WM", "D2D", "DNBR", "TM", "TD",
]

ORACLE_ERRORS = {1: "invalid input graph", 2: "out of memory", 4: "128-bit overflow"}


def build(force: bool = False, parallel: bool = False) -> str:
    """Compile escape_oracle.c into liboracle.so (plain gcc, portable flags).

    ``parallel=True`` builds liboracle_omp.so from the same source with
    -fopenmp: the census loops over vertices run on OMP_NUM_THREADS threads
    (the arithmetic is the same; only the order of exact additions differs).
    The serial build is the default and the one the pins run on."""
    lib, flags = (_LIB_OMP, ["-fopenmp"]) if parallel else (_LIB, [])
    if force or not os.path.exists(lib) or os.path.getmtime(lib) < os.path.getmtime(_SRC):
        tmp = lib + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", *flags, "-shared", "-fPIC", "-o", tmp, _SRC])
        os.replace(tmp, lib)
    return lib


def _load(parallel: bool = False):
    global _lib, _lib_omp
    with _lock:
        if parallel and _lib_omp is not None:
            return _lib_omp
        if not parallel and _lib is not None:
            return _lib
        lib = ctypes.CDLL(build(parallel=parallel))
        P, i64, c_int = ctypes.c_void_p, ctypes.c_int64, ctypes.c_int
        lib.oracle_brute_census.restype = c_int
        lib.oracle_brute_census.argtypes = [i64, P, P, P, P, P]
        lib.oracle_matrix.restype = c_int
        lib.oracle_matrix.argtypes = [c_int, P]
        lib.oracle_classify.restype = c_int
        lib.oracle_classify.argtypes = [c_int, c_int]
        lib.oracle_census_sums.restype = c_int
        lib.oracle_census_sums.argtypes = [i64, P, P, P, P, P, P, P, P, P]
        lib.oracle_edge_elements.restype = c_int
        lib.oracle_edge_elements.argtypes = [i64, P, P, i64, P, P, P, P, P]
        lib.oracle_vertex_elements.restype = c_int
        lib.oracle_vertex_elements.argtypes = [i64, P, P, i64, P, P, P]
        lib.oracle_wedge_diamond_sums.restype = c_int
        lib.oracle_wedge_diamond_sums.argtypes = [i64, P, P, P]
        lib.oracle_pair_sums.restype = c_int
        lib.oracle_pair_sums.argtypes = [i64, P, P, P]
        lib.oracle_clique4_count.restype = c_int
        lib.oracle_clique4_count.argtypes = [i64, P, P, P]
        lib.oracle_clique5_count.restype = c_int
        lib.oracle_clique5_count.argtypes = [i64, P, P, P]
        lib.oracle_num_sums.restype = c_int
        lib.oracle_num_threads.restype = c_int
        assert lib.oracle_num_sums() == len(SUM_NAMES)
        if parallel:
            _lib_omp = lib
        else:
            _lib = lib
    return lib


def num_threads(parallel: bool = False) -> int:
    """Threads the census of the given build runs on (1 for the serial build)."""
    return _load(parallel).oracle_num_threads()


def _ptr(a):
    return a.ctypes.data if a is not None else None


def _csr(g):
    rp = np.ascontiguousarray(g.row_ptr, dtype=np.int64)
    col = np.ascontiguousarray(g.col, dtype=np.int32)
    if col.size == 0:
        col = np.zeros(1, dtype=np.int32)
    return rp, col


def classify(k: int, mask: int) -> int:
    """0-based class of the k-vertex graph whose pair (a<b) bits are `mask`."""
    return _load().oracle_classify(k, mask)


def matrix(k: int) -> list[list[int]]:
    """A (ncls x ncls): A[i][j] = # spanning subgraphs of class j isomorphic to class i."""
    n = NCLS[k]
    A = np.zeros(n * n, dtype=np.int64)
    rc = _load().oracle_matrix(k, A.ctypes.data)
    if rc:
        raise RuntimeError("oracle_matrix failed")
    return [[int(x) for x in A[i * n:(i + 1) * n]] for i in range(n)]


def brute_census(g) -> dict:
    """Induced counts of every 3-, 4-, 5-vertex class by enumerating all subsets (n <= 200)."""
    rp, col = _csr(g)
    c3 = np.zeros(4, dtype=np.uint64)
    c4 = np.zeros(11, dtype=np.uint64)
    c5 = np.zeros(34, dtype=np.uint64)
    rc = _load().oracle_brute_census(g.n, rp.ctypes.data, col.ctypes.data, c3.ctypes.data,
                                     c4.ctypes.data, c5.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    return {"c3": [int(x) for x in c3], "c4": [int(x) for x in c4], "c5": [int(x) for x in c5]}


def raw_sums(g, per_element: bool = False, parallel: bool = False):
    """The C oracle's sums (Python ints), optionally with the per-element arrays."""
    rp, col = _csr(g)
    nnz = int(rp[-1]) if g.n > 0 else 0
    sums = np.zeros(2 * len(SUM_NAMES), dtype=np.uint64)
    arrs = None
    if per_element:
        arrs = {
            "T_e": np.zeros(max(nnz, 1), dtype=np.uint64),
            "t_i": np.zeros(max(g.n, 1), dtype=np.uint64),
            "C4_e": np.zeros(max(nnz, 1), dtype=np.uint64),
            "C4_i": np.zeros(max(g.n, 1), dtype=np.uint64),
            "K4_e": np.zeros(max(nnz, 1), dtype=np.uint64),
            "K4_i": np.zeros(max(g.n, 1), dtype=np.uint64),
        }
    a = arrs or {}
    rc = _load(parallel).oracle_census_sums(
        g.n, rp.ctypes.data, col.ctypes.data, sums.ctypes.data,
        _ptr(a.get("T_e")), _ptr(a.get("t_i")), _ptr(a.get("C4_e")), _ptr(a.get("C4_i")),
        _ptr(a.get("K4_e")), _ptr(a.get("K4_i")))
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    S = {name: int(sums[2 * k]) | (int(sums[2 * k + 1]) << 64) for k, name in enumerate(SUM_NAMES)}
    if arrs is not None:
        arrs = {k: (v[:nnz] if k.endswith("_e") else v[:g.n]) for k, v in arrs.items()}
        return S, arrs
    return S


def noninduced_from_sums(S: dict) -> dict:
    """Non-induced counts N (3-, 4-, 5-vertex, catalogue order) from the raw sums.

    Connected 5-vertex patterns: Thm 8 (cut = vertex: N1, N3, N4, N7, N9, N15),
    Thm 9 (cut = edge: N2, N5, N6, N11, N12, N14, N19), Thm 10 (cut = triangle:
    N10, N16, N20), Thm 11 (cut = pair/wedge: N13, N17, N18), Thm 13 (N8),
    Thm 14 (N21).  Disconnected patterns: Thm 3 (App. A).  4-vertex: Thms 4-6.
    """
    n, m, W, T = S["n"], S["m"], S["W"], S["T"]
    TT, C4, D, K4 = S["TT"], S["C4"], S["D"], S["K4"]
    S3 = S["S3"]
    P4 = S["EDGE_DD"] - 3 * T                                   # 3-paths (Thm 4)
    N = [0] * 35                                                # 1-based
    N[1] = S["S4"]
    N[2] = S["N2A"] - 2 * TT
    N[3] = S["N3A"] - 4 * C4 - 2 * TT - 3 * T
    N[4] = S["N4"]
    N[5] = S["N5A"] - 4 * D
    N[6] = S["N6A"] - 2 * D
    N[7] = S["N7A"] - 2 * D
    N[8] = S["N8M"] - S["N8Z"]
    N[9] = S["N9A"] - 2 * D
    N[10] = S["N10A"] - 12 * K4
    N[11] = S["N11"]
    N[12] = S["N12A"] - 4 * D
    N[13] = S["N13"]
    N[14] = S["N14"]
    N[15] = S["N15"]
    N[16] = S["N16A"] - 12 * K4
    N[17] = S["N17"]
    assert S["N18X4"] % 4 == 0
    N[18] = S["N18X4"] // 4
    N[19] = S["N19"]
    N[20] = S["N20"]
    N[21] = S["N21"]
    # disconnected 5-vertex patterns (Thm 3): products of connected counts
    # minus the maps that merge vertices of different components
    N[22] = comb(n, 5)
    N[23] = m * comb(n - 2, 3) if n >= 2 else 0
    N[24] = (comb(m, 2) - W) * (n - 4) if n >= 4 else 0
    N[25] = W * comb(n - 3, 2) if n >= 3 else 0
    N[26] = T * comb(n - 3, 2) if n >= 3 else 0
    N[27] = S3 * (n - 4) if n >= 4 else 0
    N[28] = P4 * (n - 4) if n >= 4 else 0
    N[29] = TT * (n - 4) if n >= 4 else 0
    N[30] = C4 * (n - 4) if n >= 4 else 0
    N[31] = D * (n - 4) if n >= 4 else 0
    N[32] = K4 * (n - 4) if n >= 4 else 0
    N[33] = S["WM"] - S["D2D"] - S["DNBR"] + 2 * W + 3 * T
    N[34] = S["TM"] - S["TD"] + 3 * T
    n5 = N[1:35]
    n4 = [S3, P4, TT, C4, D, K4, comb(n, 4), m * comb(n - 2, 2) if n >= 2 else 0,
          comb(m, 2) - W, W * (n - 3) if n >= 3 else 0, T * (n - 3) if n >= 3 else 0]
    n3 = [comb(n, 3), m * (n - 2) if n >= 2 else 0, W, T]
    return {"n3": n3, "n4": n4, "n5": n5}


def _solve_unitriangular(A: list[list[int]], N: list[int]) -> list[int]:
    """Exact solution of A C = N.  A[i][j] != 0 only when class i is a spanning
    subgraph of class j (fewer edges, or i == j with A[i][i] = 1), so solving
    from the densest class down is plain back-substitution in Python ints.
    Class j has sum_i A[i][j] = 2^(edges of j) spanning subgraphs."""
    k = len(A)
    edges = [(sum(A[i][j] for i in range(k))).bit_length() - 1 for j in range(k)]
    C = [0] * k
    for i in sorted(range(k), key=lambda c: -edges[c]):
        assert A[i][i] == 1
        C[i] = N[i] - sum(A[i][j] * C[j] for j in range(k) if j != i and A[i][j])
    return C


def induced_from_noninduced(Nd: dict) -> dict:
    out = {}
    for k, key in ((3, "n3"), (4, "n4"), (5, "n5")):
        A = matrix(k)
        out["c%d" % k] = _solve_unitriangular(A, Nd[key])
    return out


def census(g, per_element: bool = False, parallel: bool = False) -> dict:
    """Full census by the paper's method: induced (c3, c4, c5) and non-induced
    (n3, n4, n5) counts as Python ints; optionally the per-element arrays.
    ``parallel=True`` runs the OpenMP build of the same source."""
    if per_element:
        S, arrs = raw_sums(g, True, parallel)
    else:
        S, arrs = raw_sums(g, False, parallel), None
    Nd = noninduced_from_sums(S)
    out = dict(Nd)
    out.update(induced_from_noninduced(Nd))
    out["sums"] = S
    if arrs is not None:
        out["per_element"] = arrs
    return out


def wedge_diamond_sums(g, parallel: bool = False) -> dict:
    """W (wedges), T (triangles) and D (diamonds, sum over edges of C(T(e), 2))
    from their definitions, without the rest of the census."""
    rp, col = _csr(g)
    out = np.zeros(6, dtype=np.uint64)
    rc = _load(parallel).oracle_wedge_diamond_sums(g.n, rp.ctypes.data, col.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    vals = [int(out[2 * k]) | (int(out[2 * k + 1]) << 64) for k in range(3)]
    return dict(zip(("W", "T", "D"), vals))


def pair_sums(g, parallel: bool = False) -> dict:
    """C4 (4-cycles) and N13 (non-induced K2,3) from the two-hop pair counts
    W(i,j) = |N(i) cap N(j)|, without the rest of the census."""
    rp, col = _csr(g)
    out = np.zeros(4, dtype=np.uint64)
    rc = _load(parallel).oracle_pair_sums(g.n, rp.ctypes.data, col.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    vals = [int(out[2 * k]) | (int(out[2 * k + 1]) << 64) for k in range(2)]
    return dict(zip(("C4", "N13"), vals))


def clique4_count(g, parallel: bool = False) -> int:
    """The number of 4-cliques, each counted once at its lowest vertex in the
    degree order as a triangle of G[N+(x)], without the rest of the census."""
    rp, col = _csr(g)
    out = np.zeros(2, dtype=np.uint64)
    rc = _load(parallel).oracle_clique4_count(g.n, rp.ctypes.data, col.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    return int(out[0]) | (int(out[1]) << 64)


def clique5_count(g, parallel: bool = False) -> int:
    """The number of 5-cliques, each counted once at its lowest vertex in the
    degree order as a 4-clique of G[N+(x)] (bit sets and popcounts), without
    the rest of the census."""
    rp, col = _csr(g)
    out = np.zeros(2, dtype=np.uint64)
    rc = _load(parallel).oracle_clique5_count(g.n, rp.ctypes.data, col.ctypes.data, out.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    return int(out[0]) | (int(out[1]) << 64)


def edge_elements(g, us, vs) -> dict:
    """T, K4 and C4 of the given edges (u, v), each from its definition."""
    rp, col = _csr(g)
    us = np.ascontiguousarray(np.asarray(us, dtype=np.int64))
    vs = np.ascontiguousarray(np.asarray(vs, dtype=np.int64))
    k = us.size
    T = np.zeros(max(k, 1), dtype=np.uint64)
    K4 = np.zeros(max(k, 1), dtype=np.uint64)
    C4 = np.zeros(max(k, 1), dtype=np.uint64)
    rc = _load().oracle_edge_elements(g.n, rp.ctypes.data, col.ctypes.data, k, us.ctypes.data, vs.ctypes.data,
                                      T.ctypes.data, K4.ctypes.data, C4.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    return {"T_e": T[:k], "K4_e": K4[:k], "C4_e": C4[:k]}


def vertex_elements(g, vs) -> dict:
    """t and C4 of the given vertices, each from its definition."""
    rp, col = _csr(g)
    vs = np.ascontiguousarray(np.asarray(vs, dtype=np.int64))
    k = vs.size
    t = np.zeros(max(k, 1), dtype=np.uint64)
    C4 = np.zeros(max(k, 1), dtype=np.uint64)
    rc = _load().oracle_vertex_elements(g.n, rp.ctypes.data, col.ctypes.data, k, vs.ctypes.data,
                                        t.ctypes.data, C4.ctypes.data)
    if rc:
        raise ValueError(ORACLE_ERRORS.get(rc, f"oracle error {rc}"))
    return {"t_i": t[:k], "C4_i": C4[:k]}
