"""Host logic of bench.py that needs no GPU: the digest that ties a stored ncu
traffic figure to the kernel it was measured on."""
import os
import shutil

import bench


def _copy_source(tmp_path):
    src = os.path.join(bench.ROOT, "paper_1610_09411_gb300", "csrc", "census.cu")
    dst_dir = tmp_path / "paper_1610_09411_gb300" / "csrc"
    dst_dir.mkdir(parents=True)
    shutil.copy(src, dst_dir / "census.cu")
    return dst_dir / "census.cu"


def test_kernel_digest_covers_the_kernel_only(tmp_path, monkeypatch):
    path = _copy_source(tmp_path)
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    base = bench.source_digest("k_pairs")
    text = path.read_text()
    # an edit outside the kernel, its counters and its launch lines: same digest
    path.write_text(text + "\n// a note at the end of the file\n")
    assert bench.source_digest("k_pairs") == base
    # an edit inside the kernel's body: a different digest
    sig = text.index(" k_pairs(")
    body = text.index("{", sig)
    path.write_text(text[:body + 1] + "\n  // changed\n" + text[body + 1:])
    assert bench.source_digest("k_pairs") != base
    # an edit of its launch configuration: a different digest
    path.write_text(text.replace("static constexpr int PAIR_CTAS_PER_SM = 3;", "static constexpr int PAIR_CTAS_PER_SM = 2;"))
    assert bench.source_digest("k_pairs") != base

