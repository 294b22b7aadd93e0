"""Run-time model of the census from its basis counts.

The paper (Sec. 8, the runtime-prediction figure) fits the run time of its
5-vertex census to a linear function of four counts: wedges W, diamonds D,
directed 3-paths DP and directed bipyramids DBP -- the terms of Thm 2's bound
O(W + D + DP + DBP + m + n) -- with no m or n term.  This module fits the same
form to this library's GPU time,

    basis model:  t = c0 + cW W + cD D + cDP DP + cDBP DBP,

and a second form from counts the host reads off the CSR before any GPU work,

    host model:   t = c0 + cW W + cDP DP + cm m,

which the serving loop uses to size batches and to order waiting work.  Both
are non-negative least-squares fits of relative error (every graph weighs the
same whatever its size).  W, D, DP and DBP of a counted graph come from
escape_last_basis_counts; host_counts computes W and DP from the degrees.

    python -m paper_1610_09411_gb300.predict --measure   # time a family of graphs (GPU)
    python -m paper_1610_09411_gb300.predict --fit       # refit from the stored timings

Timings and coefficients are stored in predict_fit.json beside this file.
"""
from __future__ import annotations

import json
import os
import sys

import numpy as np

HERE = os.path.dirname(os.path.abspath(__file__))
FIT_PATH = os.path.join(HERE, "predict_fit.json")

MODELS = {
    "basis": ["W", "D", "DP", "DBP"],
    "host": ["W", "DP", "m"],
}


def host_counts(row_ptr, col) -> dict:
    """W = sum_i C(d_i, 2) and DP = sum over out-edges a -> b of the
    degree-ordered DAG of (d+(a) - 1) d+(b) (order by degree, ties by id,
    Sec. 3.2), from the CSR alone; plus n and m."""
    row_ptr = np.asarray(row_ptr, dtype=np.int64)
    col = np.asarray(col, dtype=np.int64)
    n = len(row_ptr) - 1
    if n <= 0 or col.size == 0:
        return {"n": max(n, 0), "m": 0, "W": 0, "DP": 0}
    deg = np.diff(row_ptr)
    src = np.repeat(np.arange(n, dtype=np.int64), deg)
    up = (deg[src] < deg[col]) | ((deg[src] == deg[col]) & (src < col))      # src precedes col
    dplus = np.bincount(src[up], minlength=n).astype(np.int64)
    W = int((deg * (deg - 1) // 2).sum())
    DP = int(((dplus[src[up]] - 1) * dplus[col[up]]).sum())
    return {"n": n, "m": int(col.size // 2), "W": W, "DP": DP}


def _design(samples, feats):
    X = np.array([[1.0] + [float(s[f]) for f in feats] for s in samples])
    t = np.array([float(s["seconds"]) for s in samples])
    return X, t


def fit(samples, feats) -> list:
    """Non-negative coefficients [c0, c_f...] minimising the relative error."""
    from scipy.optimize import nnls
    X, t = _design(samples, feats)
    w = 1.0 / t
    scale = np.maximum(np.abs(X).max(axis=0), 1e-300)        # column scaling keeps nnls well conditioned
    coef, _ = nnls((X * w[:, None]) / scale, t * w)
    return [float(c) for c in coef / scale]


def predict(coef, counts: dict, feats) -> float:
    return float(coef[0] + sum(c * float(counts[f]) for c, f in zip(coef[1:], feats)))


def held_out_error(samples, feats) -> dict:
    """Fit on the even-indexed samples, report |predicted / measured - 1| on
    the odd-indexed ones."""
    train, test = samples[0::2], samples[1::2]
    coef = fit(train, feats)
    err = [abs(predict(coef, s, feats) / s["seconds"] - 1.0) for s in test]
    return {"median": float(np.median(err)), "p90": float(np.percentile(err, 90)), "max": float(max(err)),
            "train": len(train), "test": len(test)}


def load_fit(path: str = FIT_PATH):
    try:
        with open(path) as f:
            return json.load(f)
    except OSError:
        return None


class Predictor:
    """Seconds of one census from the host counts of its CSR (host model of
    the stored fit); None coefficients (no stored fit) predict from m alone."""

    def __init__(self, fit_record=None):
        rec = fit_record if fit_record is not None else load_fit()
        self.coef = rec["models"]["host"]["coef"] if rec else None

    def seconds(self, counts: dict) -> float:
        if self.coef is None:
            return 1e-3 + 2e-8 * counts.get("m", 0)
        return predict(self.coef, counts, MODELS["host"])


# ---------------------------------------------------------------- measurement (GPU)

def family():
    """Graphs of the kinds the workloads use, over a range of sizes."""
    import graphgen as gg
    out = []
    for k, (n, p) in enumerate([(2000, 0.01), (5000, 0.004), (20000, 0.0008), (1000, 0.1), (1500, 0.2),
                                (2000, 0.3), (800, 0.25), (50000, 0.0003)]):
        out.append(gg.erdos_renyi(n, p, 10 + k))
    for k, (n, m) in enumerate([(5000, 3), (20000, 5), (100000, 4), (300000, 6), (2000, 2)]):
        out.append(gg.barabasi_albert(n, m, 20 + k))
    for k, (n, gam, md) in enumerate([(20000, 2.1, 12), (65536, 2.1, 16), (262144, 2.1, 16), (100000, 2.3, 16),
                                      (400000, 2.3, 8), (30000, 2.5, 20), (150000, 2.1, 24)]):
        out.append(gg.chung_lu(n, gam, md, min(8192.0, n / 4), 30 + k))
    for k, sc in enumerate([14, 15, 16, 17, 18, 19, 20]):
        out.append(gg.config_rmat(sc, 40 + k))
    for k in range(6):
        out.append(gg.batch_member(100 + 37 * k, 2024))
    return out


def measure(graphs, reps: int = 3):
    """GPU seconds (best of reps, CUDA events around the census call) and the
    counts of every graph."""
    import torch
    from . import escape as esc
    samples = []
    for g in graphs:
        rp = torch.from_numpy(g.row_ptr).cuda()
        col = torch.from_numpy(g.col if g.col.size else np.zeros(1, np.int32)).cuda()
        torch.cuda.synchronize()
        h = esc.escape_load_csr(g.n, rp, col[:g.nnz])
        try:
            esc.escape_census5(h)                                 # warm-up
            best = None
            for _ in range(reps):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                st = torch.cuda.current_stream()
                e0.record(st)
                esc.escape_census5(h)
                e1.record(st)
                e1.synchronize()
                ms = e0.elapsed_time(e1)
                best = ms if best is None else min(best, ms)
            basis = esc.escape_last_basis_counts(h)
        finally:
            esc.escape_free(h)
        s = {"graph": g.name, "seconds": best / 1000.0}
        s.update(host_counts(g.row_ptr, g.col))
        s.update({k: int(v) for k, v in basis.items()})
        samples.append(s)
        print(json.dumps(s), flush=True)
    return samples


def fit_record(samples) -> dict:
    rec = {"samples": samples, "models": {}}
    for name, feats in MODELS.items():
        rec["models"][name] = {"features": ["1"] + feats, "coef": fit(samples, feats),
                               "held_out": held_out_error(samples, feats)}
    return rec


def main(argv):
    if "--measure" in argv:
        root = os.path.dirname(HERE)
        if root not in sys.path:
            sys.path.insert(0, root)
        import torch
        torch.cuda.set_device(0)
        samples = measure(family())
        rec = fit_record(samples)
    elif "--fit" in argv:
        rec = fit_record(load_fit()["samples"])
    else:
        print(__doc__)
        return
    with open(FIT_PATH, "w") as f:
        json.dump(rec, f, indent=1)
    for name, m in rec["models"].items():
        print(name, "held-out relative error", m["held_out"])


if __name__ == "__main__":
    main(sys.argv[1:])
