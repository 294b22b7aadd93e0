"""Host logic of the autotuner: size classes, applying and clearing the stored
knobs of a class (the tuning itself needs a GPU and is checked there: every
knob value gives the same counts)."""
import os

from paper_1610_09411_gb300 import autotune as at


def test_size_classes():
    assert at.size_class(0) == "small"
    assert at.size_class((1 << 18) - 1) == "small"
    assert at.size_class(1 << 18) == "medium"
    assert at.size_class(3_933_078) == "medium"          # the Chung-Lu workload
    assert at.size_class(31_403_380) == "large"         # R-MAT scale 20
    assert at.size_class(128_301_698) == "huge"         # R-MAT scale 22


def test_apply_sets_and_clears_the_class_knobs(monkeypatch):
    for k in at.KNOBS:
        monkeypatch.delenv(k, raising=False)
    table = {"huge": {"ESC_PAIR_CLUSTER": 8, "ESC_PAIR_SHAPE": 3, "ms": 1.0, "graph": "x"},
             "medium": {"ESC_CTA_PER_SM": 3}}
    got = at.apply(128_301_698, table)
    assert got == {"ESC_PAIR_CLUSTER": 8, "ESC_PAIR_SHAPE": 3}
    assert os.environ["ESC_PAIR_CLUSTER"] == "8" and os.environ["ESC_PAIR_SHAPE"] == "3"
    assert at.cta_per_sm() == 0
    at.apply(3_933_078, table)
    assert "ESC_PAIR_CLUSTER" not in os.environ and at.cta_per_sm() == 3
    at.apply(10, table)
    assert all(k not in os.environ for k in at.KNOBS)


def test_every_knob_value_is_in_the_library_range():
    assert set(at.KNOBS["ESC_PAIR_CLUSTER"]) <= {1, 2, 4, 8, 16}
    assert set(at.KNOBS["ESC_PAIR_WINDOW"]) <= {1, 2, 3}
    assert set(at.KNOBS["ESC_PAIR_SHAPE"]) <= {1, 2, 3}
    assert max(at.KNOBS["ESC_WHEEL_WARP_MAX"]) <= 1024 and max(at.KNOBS["ESC_CLQ_WARP_DIN"]) <= 512
    assert set(at.KNOBS["ESC_CTA_PER_SM"]) <= set(range(1, 9))
