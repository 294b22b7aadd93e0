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
    # an edit of another sweep: same digest
    w = text.index("k_wheels_cta(")
    path.write_text(text[:w] + "/* other */ " + text[w:])
    assert bench.source_digest("k_pairs") == base
    # an edit inside a pair-sweep kernel's body: a different digest
    sig = text.index(" k_pairs_grp(")
    body = text.index("{", sig)
    path.write_text(text[:body + 1] + "\n  // changed\n" + text[body + 1:])
    assert bench.source_digest("k_pairs") != base
    # an edit of its launch configuration: a different digest
    old = "static constexpr int PAIR_TASK = 32 * 4 * 4;"
    assert old in text
    path.write_text(text.replace(old, "static constexpr int PAIR_TASK = 32 * 4 * 8;"))
    assert bench.source_digest("k_pairs") != base
    plan = "const size_t budget = (size_t)std::max(l2, 1 << 20) / 2;"
    assert plan in text
    path.write_text(text.replace(plan, plan.replace("/ 2", "/ 3")))
    assert bench.source_digest("k_pairs") != base

