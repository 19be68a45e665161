"""Autotuner host logic (CPU) and one tuning pass on the GPU."""
import pytest

from paper_2507_02164_gb300 import autotune


def test_choose_groups_sums_over_each_group():
    tables = {
        2: {(64, 0): 1.0, (128, 0): 2.0},
        6: {(64, 0): 5.0, (128, 0): 3.5},
        8: {(128, 0): 7.0, (256, 1): 6.0},
        12: {(256, 1): 9.0, (128, 0): 9.5},
    }
    g = autotune.choose_groups(tables)
    # group 1-6: (64, 0) sums 1 + 5 = 6.0, (128, 0) sums 2 + 3.5 = 5.5 -> (128, 0)
    assert g[0] == [128, 0]
    assert g[1] == [256, 1]
    assert g[2] == [256, 1]


def test_choose_groups_without_degrees_gives_defaults():
    assert autotune.choose_groups({3: {(64, 2): 1.0}}) == [[64, 2], [0, 0], [0, 0]]


@pytest.mark.gpu
def test_tune_two_degrees_on_gpu(tmp_path):
    from tests.gpu_common import require_gpu
    require_gpu()
    res = autotune.tune("mixed", degrees=(3, 6), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert set(res["degrees"]) == {"3", "6"}
    for e in res["degrees"].values():
        assert e["block"] in autotune.BLOCKS and e["ms"] > 0
    # a later request for more degrees measures only the new one
    more = autotune.tune("mixed", degrees=(3, 6, 9), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert more["degrees"]["3"] == res["degrees"]["3"] and "9" in more["degrees"]
    again = autotune.tune("mixed", degrees=(3, 6, 9), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert again["degrees"] == more["degrees"] and again["groups"] == more["groups"]
