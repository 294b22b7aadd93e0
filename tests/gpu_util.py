"""Helpers for the GPU parity tests (import only from tests)."""
import numpy as np


def gpu_census(g, per_element=False, device=False, flags=0):
    from paper_1610_09411_gb300 import escape as esc
    if device:
        import torch
        rp = torch.from_numpy(g.row_ptr).cuda()
        col = torch.from_numpy(g.col if g.col.size else np.zeros(1, np.int32)).cuda()
        if g.col.size == 0:
            col = col[:0]
        torch.cuda.synchronize()
        return esc.census(rp, col, n=g.n, per_element=per_element, flags=flags)
    return esc.census(g.row_ptr, g.col, n=g.n, per_element=per_element, flags=flags)


def assert_same_census(got, want, keys=("c3", "c4", "c5", "n3", "n4", "n5")):
    for k in keys:
        assert got[k] == want[k], (k, [(i, a, b) for i, (a, b) in enumerate(zip(got[k], want[k])) if a != b][:6])


def graph_hash(g) -> str:
    """SHA-256 of a generated CSR (n, row_ptr, col): identifies the graph a
    stored oracle result belongs to."""
    import hashlib
    h = hashlib.sha256()
    h.update(str(g.n).encode())
    h.update(g.row_ptr.astype("<i8").tobytes())
    h.update(g.col.astype("<i4").tobytes())
    return h.hexdigest()
