"""A census split over parts (owner ranges of the work items), on one GPU:
every part counted through the C ABI on its own handle, the parts' sums and
per-element arrays added on the host, and the finish step's census equal to
the whole census and to the oracle, bit for bit."""
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


def _split_census(g, parts):
    from paper_1610_09411_gb300 import escape as esc
    handles = [esc.escape_load_csr(g.n, g.row_ptr, g.col) for _ in range(parts)]
    try:
        sums = [esc.escape_census5_part(h, p, parts) for p, h in enumerate(handles)]
        total = [sum(col) % (1 << 128) for col in zip(*sums)]
        nnz = max(g.nnz, 1)
        acc = [np.zeros(nnz, np.uint64), np.zeros(nnz, np.uint64), np.zeros(max(g.n, 1), np.uint64)]
        for h in handles:
            got = [np.zeros_like(a) for a in acc]
            esc.escape_part_counts(h, *got)
            for a, b in zip(acc, got):
                a += b
        esc.escape_part_counts(handles[0], *acc, put=True)
        return esc.escape_census5_finish(handles[0], total), sums
    finally:
        for h in handles:
            esc.escape_free(h)


@pytest.mark.parametrize("parts", [1, 2, 3])
@pytest.mark.parametrize("make", [
    lambda: gg.chung_lu(20000, 2.1, 10, 2000, 8),
    lambda: gg.barabasi_albert(3000, 5, 4),
    lambda: gg.config_er500(3),
    lambda: gg.complete(45),
    lambda: gg.config_rmat(13, 2),
    lambda: gg.disjoint_union([gg.star(500), gg.complete(30), gg.cycle(9)]),
], ids=["chung_lu", "ba", "er500", "K45", "rmat13", "union"])
def test_parts_summed_equal_the_whole_census(make, parts):
    g = make()
    got, sums = _split_census(g, parts)
    whole = gpu_census(g)
    assert_same_census(got, whole)
    assert_same_census(got, oracle.census(g))
    if parts > 1:
        # every part did some of the sweep work
        assert all(any(v for v in s) for s in sums)


def test_two_hubs_split_matches_the_stored_oracle_result():
    """Counts at the hubs above 2^16 (64-bit counter words) split in two."""
    import json
    import os
    from gpu_util import graph_hash
    path = os.path.join(os.path.dirname(__file__), "golden", "census_two_hubs.json")
    with open(path) as f:
        gold = json.load(f)
    g = gg.two_hubs()
    assert gold["sha256"] == graph_hash(g)
    got, _ = _split_census(g, 2)
    for key in ("c3", "c4", "c5", "n3", "n4", "n5"):
        assert got[key] == [int(x) for x in gold[key]], key


def test_part_arguments_checked():
    from paper_1610_09411_gb300 import escape as esc
    g = gg.complete(8)
    h = esc.escape_load_csr(g.n, g.row_ptr, g.col)
    try:
        for part, parts in ((2, 2), (-1, 2), (0, 0)):
            with pytest.raises(esc.EscapeError) as ei:
                esc.escape_census5_part(h, part, parts)
            assert ei.value.code == 1
        with pytest.raises(esc.EscapeError):          # no part held
            esc.escape_census5_finish(h, [0] * esc.escape_part_sum_count())
    finally:
        esc.escape_free(h)
