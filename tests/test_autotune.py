"""Autotuner host logic (CPU) and tuning passes through the C ABI on the GPU."""
import ctypes
import os

import pytest

from paper_2507_02164_gb300 import _native as N
from paper_2507_02164_gb300 import autotune, build


def test_uneven_tuning_takes_the_warp_specialised_winner_up_to_degree_8_else_the_one_role_one():
    ws = {"lanes": 1, "block": 512, "ctas_per_sm": 0, "polish_warps": 10, "ms": 1.0,
          "one_role": {"lanes": 1, "block": 256, "ctas_per_sm": 2, "ms": 1.1}}
    res = {"degrees": {"6": dict(ws), "9": dict(ws, block=256, polish_warps=4)}}
    t = autotune.uneven_tuning(res)
    assert list(t.block)[6] == 512 and list(t.polish_warps)[6] == 10 and list(t.ctas_per_sm)[6] == 0
    assert list(t.block)[9] == 256 and list(t.polish_warps)[9] == 0 and list(t.ctas_per_sm)[9] == 2
    p = autotune.degree_params(res, 6)
    assert p.block == 512 and p.polish_warps == 10


def test_uneven_tuning_is_per_degree():
    res = {"degrees": {"3": {"lanes": 1, "block": 64, "ctas_per_sm": 2},
                       "12": {"lanes": 2, "block": 128, "ctas_per_sm": 0}}}
    t = autotune.uneven_tuning(res)
    assert list(t.block)[3] == 64 and list(t.block)[12] == 128 and list(t.lanes)[12] == 2
    assert list(t.ctas_per_sm)[3] == 2 and list(t.lanes)[3] == 1
    assert sum(t.block) == 64 + 128  # other degrees left at the defaults
    with pytest.raises(ValueError):
        autotune.api.uneven_tuning(block={13: 64})


def test_source_hash_follows_every_library_source(tmp_path, monkeypatch):
    """A cached tuning is keyed on the library's sources: changing any kernel
    source, header or the C ABI header gives another key."""
    h0 = build.source_hash()
    assert h0 == build.source_hash() and len(h0) == 16
    deps = sorted(build._deps())
    assert any(p.endswith("rootdensity.h") for p in deps) and any(p.endswith("rd_solve.cuh") for p in deps)
    fake = tmp_path / "rd_extra.cu"
    fake.write_text("// one more unit\n")
    monkeypatch.setattr(build, "_deps", lambda: deps + [str(fake)])
    assert build.source_hash() != h0


@pytest.mark.gpu
def test_c_autotuner_times_every_candidate_and_picks_the_fastest():
    from tests.gpu_common import require_gpu
    require_gpu()
    L = N.load()
    for degree, mode, polish in ((6, N.MIXED, N.POLISH_FP64), (9, N.MIXED, N.POLISH_FP64), (6, N.PLAIN_FP64, 0),
                                 (6, N.MIXED, N.POLISH_DF)):
        t = N.Tuning()
        tab = (N.TuneEntry * 64)()
        used = ctypes.c_int(0)
        rc = L.rd_autotune(degree, mode, polish, N.C64 if mode == N.MIXED else N.C128, 1 << 14, 3, ctypes.byref(t),
                           tab, 64, ctypes.byref(used))
        assert rc == 0, L.rd_last_error()
        rows = list(tab[:used.value])
        assert used.value == t.n_candidates >= 12
        ok = [r for r in rows if r.ms >= 0]
        assert ok and all(r.ms > 0 for r in ok)
        fastest = min(r.ms for r in ok)
        assert t.best.ms == fastest
        assert t.one_role.polish_warps == 0 and t.one_role.ms == min(r.ms for r in ok if r.polish_warps == 0)
        ws = [r for r in rows if r.polish_warps > 0]
        assert (len(ws) > 0) == (mode == N.MIXED)
        for r in ws:
            assert r.lanes == 1 and r.block % 32 == 0 and 1 <= r.polish_warps < r.block // 32
            assert r.block <= (512 if degree <= 6 else 256)
        assert {r.lanes for r in rows} == ({1} if polish == N.POLISH_DF else {1, 2})
    # a table smaller than the candidate list keeps the first entries
    t = N.Tuning()
    tab = (N.TuneEntry * 4)()
    used = ctypes.c_int(0)
    assert L.rd_autotune(3, N.MIXED, N.POLISH_FP64, N.C64, 1 << 12, 1, ctypes.byref(t), tab, 4,
                         ctypes.byref(used)) == 0
    assert used.value == 4 and t.n_candidates > 4


@pytest.mark.gpu
def test_tune_two_degrees_on_gpu(tmp_path):
    from tests.gpu_common import require_gpu
    require_gpu()
    res = autotune.tune("mixed", degrees=(3, 6), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert set(res["degrees"]) == {"3", "6"}
    for d, e in res["degrees"].items():
        assert e["ms"] > 0 and e["one_role"]["ms"] >= e["ms"]
        assert e["one_role"]["block"] in (32, 64, 128, 256)
        assert [e["lanes"], e["block"], e["ctas_per_sm"], e["polish_warps"], e["ms"]] in e["table"]
    # a later request for more degrees measures only the new one
    more = autotune.tune("mixed", degrees=(3, 6, 9), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert more["degrees"]["3"] == res["degrees"]["3"] and "9" in more["degrees"]
    again = autotune.tune("mixed", degrees=(3, 6, 9), n=1 << 14, cache_path=str(tmp_path / "t.json"))
    assert again["degrees"] == more["degrees"]
    assert {e["lanes"] for e in again["degrees"].values()} <= {1, 2}
    assert os.path.exists(tmp_path / "t.json")
