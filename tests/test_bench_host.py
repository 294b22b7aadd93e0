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



def test_stored_oracle_runs_and_traffic_record():
    """The CPU-baseline context and the roofline's traffic come from committed
    files: the R-MAT 22 workload has no stored full census, so its baseline
    points at the stored R-MAT 20 run; the traffic record carries the digest of
    the kernel source it was taken on (the bench reports it only while that
    digest is current)."""
    import json
    assert bench.stored_oracle_run("rmat22") is None
    rel = bench.stored_oracle_run(bench.RELATED_FULL["rmat22"][0])
    assert rel is not None and rel["seconds"] > 0 and rel["m"] > 0
    with open(os.path.join(bench.ROOT, "profiles", "traffic.json")) as f:
        rec = json.load(f)["k_pairs:rmat22"]
    assert rec["dram_bytes_per_launch"] > 0 and len(rec["source_sha"]) == 16
    current = bench.stored_traffic("k_pairs", "rmat22")
    assert current in (None, rec["dram_bytes_per_launch"])
    assert bench.stored_traffic("k_pairs", "no_such_workload") is None


def test_byte_model_sums_come_from_the_stored_oracle():
    """W and D of the byte model are read from the stored oracle sums of the
    workload graph (matched by the CSR hash)."""
    import json
    with open(os.path.join(bench.ROOT, "tests", "golden", "sums_rmat22.json")) as f:
        gold = json.load(f)
    assert {"W", "T", "D"} <= set(gold["sums"])
    assert gold["n"] == 4194304
