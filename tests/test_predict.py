"""Run-time model (the paper's fit of census time to its basis counts): the
host counts against their definitions, the fit on synthetic data with a known
answer, and the stored GPU timings (predict_fit.json) refit with the stated
held-out error."""
import itertools
import os

import numpy as np
import pytest

import graphgen as gg
from paper_1610_09411_gb300 import predict as pr


def _brute_dp(g):
    """Directed 3-paths i <- a -> b -> j with i != b (j may equal i), by
    enumeration in the degree order (ties by id)."""
    deg = g.degrees()
    prec = lambda a, b: (deg[a], a) < (deg[b], b)
    out = {v: [u for u in g.col[g.row_ptr[v]:g.row_ptr[v + 1]] if prec(v, u)] for v in range(g.n)}
    cnt = 0
    for a in range(g.n):
        for b in out[a]:
            for i in out[a]:
                if i == b:
                    continue
                cnt += len(out[b])
    return cnt


@pytest.mark.parametrize("g", [gg.erdos_renyi(40, 0.2, 1), gg.barabasi_albert(60, 3, 2), gg.complete(9),
                               gg.star(12), gg.empty(5), gg.chung_lu(200, 2.1, 6, 40, 3)], ids=lambda g: g.name)
def test_host_counts_match_definitions(g):
    c = pr.host_counts(g.row_ptr, g.col)
    deg = g.degrees()
    assert c["W"] == sum(int(d) * (int(d) - 1) // 2 for d in deg)
    assert c["DP"] == _brute_dp(g)
    assert c["m"] == g.m and c["n"] == g.n


def test_fit_recovers_a_known_linear_model():
    rng = np.random.default_rng(5)
    true = [2e-3, 3e-10, 0.0, 5e-11, 1e-12]               # c0, W, D, DP, DBP
    samples = []
    for _ in range(30):
        s = {"W": int(rng.integers(1e6, 1e10)), "D": int(rng.integers(1e6, 1e11)),
             "DP": int(rng.integers(1e6, 1e12)), "DBP": int(rng.integers(1e3, 1e12))}
        s["seconds"] = true[0] + sum(c * s[f] for c, f in zip(true[1:], pr.MODELS["basis"]))
        samples.append(s)
    coef = pr.fit(samples, pr.MODELS["basis"])
    for c, t in zip(coef, true):
        assert abs(c - t) <= 1e-6 * max(t, 1e-9) + 1e-15
    assert pr.held_out_error(samples, pr.MODELS["basis"])["max"] < 1e-6


def test_stored_gpu_timings_refit():
    rec = pr.load_fit()
    if rec is None:
        pytest.skip("no stored timings")
    samples = rec["samples"]
    assert len(samples) >= 20
    for name, feats in pr.MODELS.items():
        coef = pr.fit(samples, feats)
        assert np.allclose(coef, rec["models"][name]["coef"], rtol=1e-6, atol=1e-18)
        err = pr.held_out_error(samples, feats)
        assert err == pytest.approx(rec["models"][name]["held_out"])
        assert all(c >= 0 for c in coef)
    # the predictor the serving loop uses reads the host model
    p = pr.Predictor(rec)
    s0 = samples[0]
    assert p.seconds(s0) == pytest.approx(pr.predict(rec["models"]["host"]["coef"], s0, pr.MODELS["host"]))
