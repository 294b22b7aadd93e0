"""escape_cycles4_noalloc: per-vertex 4-cycle counts with no allocation in the
library (for callers that cannot allocate device memory when they count).

Checked through the C ABI against the existing census entry point
(escape_census5 + escape_per_element) and against the CPU oracle, on two
calls in a row so that the shared fixed work space is shown to start clean
each time, and with the device's free memory unchanged across the second
call.  Collected last on purpose; it must also pass alone in a fresh process.
"""
import numpy as np
import pytest

import graphgen as gg
import oracle

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no GPU")
    torch.cuda.set_device(0)
    from paper_1610_09411_gb300 import build
    build.build()


def _reference(g):
    from paper_1610_09411_gb300 import escape as esc
    r = esc.census(g.row_ptr, g.col, n=g.n, per_element=True)
    return r["per_element"]["C4_i"], r["n4"][3]


@pytest.mark.parametrize("make", [
    lambda: gg.erdos_renyi(300, 0.05, 1),
    lambda: gg.barabasi_albert(2000, 4, 2),
    lambda: gg.chung_lu(5000, 2.1, 10, 500, 3),
    lambda: gg.complete(40),
    lambda: gg.chung_lu(32768, 2.1, 16, 8192, 4),      # exactly the maximum size
], ids=["er300", "ba2000", "cl5000", "K40", "cl_max"])
def test_noalloc_matches_census_on_two_calls(make):
    import torch
    from paper_1610_09411_gb300 import escape as esc
    g = make()
    want_v, want_total = _reference(g)
    o = oracle.census(g, per_element=True)
    assert np.array_equal(o["per_element"]["C4_i"], want_v) and o["n4"][3] == want_total
    rp = torch.from_numpy(g.row_ptr).cuda()
    col = torch.from_numpy(g.col).cuda()
    for call in range(2):
        c4_v = torch.full((g.n,), 7, dtype=torch.int64, device="cuda")     # garbage on purpose
        total = torch.full((1,), 7, dtype=torch.int64, device="cuda")
        torch.cuda.synchronize()
        free_before = torch.cuda.mem_get_info()[0]
        esc.escape_cycles4_noalloc(g.n, rp, col, c4_v, total)
        free_after = torch.cuda.mem_get_info()[0]
        if call == 1:       # the first call on a device may load the module that holds the array
            assert free_after == free_before
        assert np.array_equal(c4_v.cpu().numpy().astype(np.uint64), want_v)
        assert int(total.item()) == want_total


def test_noalloc_rejects_oversize_graph():
    import torch
    from paper_1610_09411_gb300 import escape as esc
    n = esc.ESCAPE_NOALLOC_MAX_N + 1
    rp = torch.zeros(n + 1, dtype=torch.int64, device="cuda")
    col = torch.zeros(1, dtype=torch.int32, device="cuda")
    out = torch.zeros(n, dtype=torch.int64, device="cuda")
    tot = torch.zeros(1, dtype=torch.int64, device="cuda")
    with pytest.raises(esc.EscapeError) as ei:
        esc.escape_cycles4_noalloc(n, rp, col, out, tot)
    assert ei.value.code == 4
