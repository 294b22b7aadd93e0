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


def gpu_batch(graphs, device=False):
    """escape_census5_batch over the block-diagonal union of `graphs`."""
    from paper_1610_09411_gb300 import escape as esc
    voff = np.zeros(len(graphs) + 1, dtype=np.int64)
    rps, cols, base = [], [], 0
    for k, g in enumerate(graphs):
        voff[k + 1] = voff[k] + g.n
        rps.append(g.row_ptr[:-1] + base)
        cols.append(g.col)
        base += g.nnz
    rp = np.concatenate(rps + [np.array([base])]).astype(np.int64)
    col = np.concatenate(cols).astype(np.int32) if cols else np.zeros(0, np.int32)
    if device:
        import torch
        return esc.escape_census5_batch(torch.from_numpy(voff).cuda(), torch.from_numpy(rp).cuda(),
                                        torch.from_numpy(col).cuda())
    return esc.escape_census5_batch(voff, rp, col)
