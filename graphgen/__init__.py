"""Seeded synthetic graphs: the one module both the CUDA path's tests/benchmark
and the oracle's tests draw their inputs from.

It contains no census arithmetic.  Graphs come back as a simple undirected CSR
``Graph(n, row_ptr:int64[n+1], col:int32[2m])`` with sorted neighbour lists,
no duplicates and no self-loops (the input convention of the paper's
experiments, Sec. 8).  The random generators live in ``graphgen.c`` (compiled
on first use); small structured graphs are built here.

Workload recipes (the synthetic stand-ins for the paper's SNAP / Network
Repository graphs):
  * ``erdos_renyi(500, 0.012, seed)``             -- small G(n, p)
  * ``chung_lu(262144, 2.1, 16, 8192, seed=1)``   -- power-law, ~2M edges
  * ``rmat(22, 16, 0.57, 0.19, 0.19, seed=1)``    -- R-MAT scale 22, ~64M edges
  * ``batch_graphs(count, seed)``                 -- half G(n, p), half BA
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading
from dataclasses import dataclass

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "graphgen.c")
_LIB = os.path.join(_HERE, "libgraphgen.so")
_lock = threading.Lock()
_lib = None


def build(force: bool = False) -> str:
    """Compile graphgen.c into libgraphgen.so (plain gcc, portable flags)."""
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < os.path.getmtime(_SRC):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-shared", "-fPIC", "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def _load():
    global _lib
    with _lock:
        if _lib is None:
            build()
            lib = ctypes.CDLL(_LIB)
            P = ctypes.c_void_p
            i64, u64, dbl = ctypes.c_int64, ctypes.c_uint64, ctypes.c_double
            lib.gg_erdos_renyi.restype = P
            lib.gg_erdos_renyi.argtypes = [i64, u64, u64]
            lib.gg_chung_lu.restype = P
            lib.gg_chung_lu.argtypes = [i64, dbl, dbl, dbl, u64]
            lib.gg_rmat.restype = P
            lib.gg_rmat.argtypes = [ctypes.c_int, i64, dbl, dbl, dbl, u64]
            lib.gg_barabasi_albert.restype = P
            lib.gg_barabasi_albert.argtypes = [i64, i64, u64]
            lib.gg_from_edges.restype = P
            lib.gg_from_edges.argtypes = [i64, i64, P, P]
            lib.gg_n.restype = i64
            lib.gg_n.argtypes = [P]
            lib.gg_nnz.restype = i64
            lib.gg_nnz.argtypes = [P]
            lib.gg_copy.restype = None
            lib.gg_copy.argtypes = [P, P, P]
            lib.gg_free.restype = None
            lib.gg_free.argtypes = [P]
            lib.gg_stream_draw.restype = u64
            lib.gg_stream_draw.argtypes = [u64, u64, u64]
            _lib = lib
    return _lib


@dataclass
class Graph:
    n: int
    row_ptr: np.ndarray  # int64[n+1]
    col: np.ndarray      # int32[nnz]
    name: str = ""

    @property
    def nnz(self) -> int:
        return int(self.row_ptr[-1]) if self.n > 0 else 0

    @property
    def m(self) -> int:
        return self.nnz // 2

    def degrees(self) -> np.ndarray:
        return np.diff(self.row_ptr)

    def edges(self):
        """Unordered edge list (u < v) as two int64 arrays."""
        src = np.repeat(np.arange(self.n, dtype=np.int64), self.degrees())
        dst = self.col.astype(np.int64)
        keep = src < dst
        return src[keep], dst[keep]


def _take(handle, name: str) -> Graph:
    lib = _load()
    if not handle:
        raise MemoryError("graph generation failed")
    n = lib.gg_n(handle)
    nnz = lib.gg_nnz(handle)
    row_ptr = np.zeros(n + 1, dtype=np.int64)
    col = np.zeros(max(nnz, 1), dtype=np.int32)
    lib.gg_copy(handle, row_ptr.ctypes.data, col.ctypes.data)
    lib.gg_free(handle)
    return Graph(int(n), row_ptr, col[:nnz].copy(), name)


def from_edges(n: int, src, dst, name: str = "") -> Graph:
    """Normalise an arbitrary edge list (either direction, duplicates and loops allowed)."""
    src = np.ascontiguousarray(np.asarray(src, dtype=np.int64))
    dst = np.ascontiguousarray(np.asarray(dst, dtype=np.int64))
    if src.shape != dst.shape:
        raise ValueError("src/dst length mismatch")
    h = _load().gg_from_edges(int(n), int(src.size), src.ctypes.data, dst.ctypes.data)
    if not h:
        raise ValueError("vertex id out of range")
    return _take(h, name)


def erdos_renyi(n: int, p: float, seed: int) -> Graph:
    thr = min(int(p * 2.0 ** 64), 2 ** 64 - 1)
    return _take(_load().gg_erdos_renyi(int(n), thr, int(seed)), f"er_n{n}_p{p}_s{seed}")


def chung_lu(n: int, gamma: float, mean_deg: float, max_deg: float, seed: int) -> Graph:
    return _take(_load().gg_chung_lu(int(n), float(gamma), float(mean_deg), float(max_deg), int(seed)),
                 f"cl_n{n}_g{gamma}_s{seed}")


def rmat(scale: int, edge_factor: int = 16, a: float = 0.57, b: float = 0.19, c: float = 0.19,
         seed: int = 1) -> Graph:
    return _take(_load().gg_rmat(int(scale), int(edge_factor), float(a), float(b), float(c), int(seed)),
                 f"rmat_s{scale}_ef{edge_factor}_s{seed}")


def barabasi_albert(n: int, m_attach: int, seed: int) -> Graph:
    return _take(_load().gg_barabasi_albert(int(n), int(m_attach), int(seed)), f"ba_n{n}_m{m_attach}_s{seed}")


def stream_draw(seed: int, stream: int, ctr: int) -> int:
    """One 64-bit draw of the counter-based stream (for seeded parameter choices)."""
    return int(_load().gg_stream_draw(int(seed) & (2 ** 64 - 1), int(stream), int(ctr)))


# ---------------------------------------------------------------- structured graphs

def empty(n: int) -> Graph:
    return from_edges(n, [], [], f"empty{n}")


def complete(n: int) -> Graph:
    i, j = np.triu_indices(n, 1)
    return from_edges(n, i, j, f"K{n}")


def star(n: int) -> Graph:
    """Star S_n: centre 0 joined to n-1 leaves."""
    return from_edges(n, np.zeros(max(n - 1, 0), dtype=np.int64), np.arange(1, n), f"star{n}")


def cycle(n: int) -> Graph:
    i = np.arange(n)
    return from_edges(n, i, (i + 1) % n, f"C{n}")


def path(n: int) -> Graph:
    i = np.arange(max(n - 1, 0))
    return from_edges(n, i, i + 1, f"P{n}")


def complete_bipartite(a: int, b: int) -> Graph:
    i, j = np.meshgrid(np.arange(a), np.arange(a, a + b), indexing="ij")
    return from_edges(a + b, i.ravel(), j.ravel(), f"K{a},{b}")


def two_hubs(leaves: int = 65600) -> Graph:
    """Two adjacent hubs 0 and 1 joined to every leaf 2 .. leaves+1, a path over
    the first 400 leaves and a clique on the next 19: two vertices of degree
    above 2^16 whose common neighbourhood also exceeds 2^16."""
    s = [np.zeros(leaves, np.int64), np.ones(leaves, np.int64), np.array([0])]
    d = [np.arange(2, leaves + 2), np.arange(2, leaves + 2), np.array([1])]
    p = np.arange(2, 401)
    s.append(p)
    d.append(p + 1)
    i, j = np.triu_indices(19, 1)
    s.append(402 + i)
    d.append(402 + j)
    return from_edges(leaves + 2, np.concatenate(s), np.concatenate(d), f"two_hubs{leaves}")


def petersen() -> Graph:
    outer = [(i, (i + 1) % 5) for i in range(5)]
    spokes = [(i, i + 5) for i in range(5)]
    inner = [(5 + i, 5 + (i + 2) % 5) for i in range(5)]
    e = np.array(outer + spokes + inner)
    return from_edges(10, e[:, 0], e[:, 1], "petersen")


def relabel(g: Graph, perm) -> Graph:
    """Graph with vertex v renamed perm[v]."""
    perm = np.asarray(perm, dtype=np.int64)
    s, d = g.edges()
    return from_edges(g.n, perm[s], perm[d], g.name + "_relabel")


def complement(g: Graph) -> Graph:
    adj = np.zeros((g.n, g.n), dtype=bool)
    s, d = g.edges()
    adj[s, d] = True
    adj[d, s] = True
    i, j = np.triu_indices(g.n, 1)
    keep = ~adj[i, j]
    return from_edges(g.n, i[keep], j[keep], g.name + "_compl")


def disjoint_union(graphs) -> Graph:
    srcs, dsts, off = [], [], 0
    for g in graphs:
        s, d = g.edges()
        srcs.append(s + off)
        dsts.append(d + off)
        off += g.n
    return from_edges(off, np.concatenate(srcs) if srcs else [], np.concatenate(dsts) if dsts else [], "union")


# ---------------------------------------------------------------- named workloads

def config_er500(seed: int = 0) -> Graph:
    """Erdos-Renyi G(n=500, p=0.012)."""
    return erdos_renyi(500, 0.012, seed)


def config_chung_lu(seed: int = 1, n: int = 262144) -> Graph:
    """Chung-Lu power law, exponent 2.1, mean degree 16, max expected degree 8192."""
    return chung_lu(n, 2.1, 16.0, 8192.0, seed)


def config_rmat(scale: int = 22, seed: int = 1) -> Graph:
    """R-MAT, edge factor 16, (a, b, c, d) = (0.57, 0.19, 0.19, 0.05)."""
    return rmat(scale, 16, 0.57, 0.19, 0.19, seed)


def batch_member(k: int, seed: int, n_lo: int = 20, n_hi: int = 2000,
                 p_lo: float = 0.01, p_hi: float = 0.3, m_lo: int = 2, m_hi: int = 6) -> Graph:
    """Graph k of the batch workload (each member is drawn from its own
    counter-based streams, so any member can be made alone): size uniform in
    [n_lo, n_hi]; even k G(n, p) with p uniform in [p_lo, p_hi], odd k
    Barabasi-Albert with m uniform in [m_lo, m_hi]."""
    n = n_lo + stream_draw(seed, 1, k) % (n_hi - n_lo + 1)
    gseed = stream_draw(seed, 2, k)
    if k % 2 == 0:
        u = (stream_draw(seed, 3, k) >> 11) / float(1 << 53)
        p = p_lo + (p_hi - p_lo) * u
        return erdos_renyi(n, p, gseed)
    m_att = m_lo + stream_draw(seed, 4, k) % (m_hi - m_lo + 1)
    return barabasi_albert(n, m_att, gseed)


def batch_graphs(count: int, seed: int, n_lo: int = 20, n_hi: int = 2000,
                 p_lo: float = 0.01, p_hi: float = 0.3, m_lo: int = 2, m_hi: int = 6):
    """`count` graphs: batch_member(0 .. count-1)."""
    return [batch_member(k, seed, n_lo, n_hi, p_lo, p_hi, m_lo, m_hi) for k in range(count)]
