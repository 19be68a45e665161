"""Autotuner host logic (CPU) and one tuning pass on the GPU."""
import pytest

from paper_2507_02164_gb300 import autotune


def test_best_shape_takes_the_fastest_with_a_stable_tie_break():
    table = {(1, 128, 0, 0): 2.0, (2, 64, 0, 0): 1.5, (2, 256, 1, 0): 1.5, (1, 64, 2, 0): 3.0}
    assert autotune.best_shape(table) == (2, 64, 0, 0)


def test_warp_specialised_candidates_fit_the_register_budget():
    for d in range(1, 13):
        for block, pw in autotune.ws_candidates(d):
            assert block % 32 == 0 and 1 <= pw < block // 32
            assert block <= (512 if d <= 6 else 256)


def test_uneven_tuning_takes_the_one_role_winner_and_uniform_params_the_overall_one():
    res = {"degrees": {"6": {"lanes": 1, "block": 512, "ctas_per_sm": 0, "polish_warps": 10, "ms": 1.0,
                             "one_role": {"lanes": 1, "block": 256, "ctas_per_sm": 2, "ms": 1.1}}}}
    t = autotune.uneven_tuning(res)
    assert list(t.block)[6] == 256 and list(t.ctas_per_sm)[6] == 2
    p = autotune.degree_params(res, 6)
    assert p.block == 512 and p.polish_warps == 10


def test_lane_candidates():
    assert autotune.lane_candidates(1) == (1,)
    assert autotune.lane_candidates(2) == (1, 2) and autotune.lane_candidates(12) == (1, 2)


def test_uneven_tuning_is_per_degree():
    res = {"degrees": {"3": {"lanes": 1, "block": 64, "ctas_per_sm": 2},
                       "12": {"lanes": 2, "block": 128, "ctas_per_sm": 0}}}
    t = autotune.uneven_tuning(res)
    assert list(t.block)[3] == 64 and list(t.block)[12] == 128 and list(t.lanes)[12] == 2
    assert list(t.ctas_per_sm)[3] == 2 and list(t.lanes)[3] == 1
    assert sum(t.block) == 64 + 128  # other degrees left at the defaults
    with pytest.raises(ValueError):
        autotune.api.uneven_tuning(block={13: 64})


@pytest.mark.gpu
def test_tune_two_degrees_on_gpu(tmp_path):
    from tests.gpu_common import require_gpu
    require_gpu()
    res = autotune.tune("mixed", degrees=(3, 6), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert set(res["degrees"]) == {"3", "6"}
    for d, e in res["degrees"].items():
        ws = {b for b, _ in autotune.ws_candidates(int(d))}
        assert (e["block"] in autotune.BLOCKS or e["block"] in ws) and e["ms"] > 0
        assert e["one_role"]["block"] in autotune.BLOCKS and e["one_role"]["ms"] >= e["ms"]
    # a later request for more degrees measures only the new one
    more = autotune.tune("mixed", degrees=(3, 6, 9), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert more["degrees"]["3"] == res["degrees"]["3"] and "9" in more["degrees"]
    again = autotune.tune("mixed", degrees=(3, 6, 9), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert again["degrees"] == more["degrees"]
    assert {e["lanes"] for e in again["degrees"].values()} <= {1, 2}
