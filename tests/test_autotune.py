"""Host-side logic of the adjoint autotuner (CPU only): candidate grid, accuracy-gated selection,
failure handling, signatures and the persistent cache.  The timed calls are faked."""
import math

import pytest

from paper_2603_16478_gb300 import autotune as at


def test_default_candidates_cover_every_variant_and_restart():
    c = at.default_candidates(451)
    assert len(c) == 3 * 3
    assert {(x["precision"], x["cap_precision"]) for x in c} == set(at.PRECISION_VARIANTS)
    assert {x["restart"] for x in c} == {32, 64, 128} and {x["cap_block"] for x in c} == {0}
    big = at.default_candidates(2329)
    assert len(big) == 3 * 3 * 2 and {x["cap_block"] for x in big} == {0, 1024}


def test_select_takes_the_fastest_accurate_success():
    trials = [at.Trial({"i": 0}, 5.0, 0.0), at.Trial({"i": 1}, 2.0, 5e-3), at.Trial({"i": 2}, 3.0, 1e-4),
              at.Trial({"i": 3}, 1.0, 0.0, error="NOT_CONVERGED"), at.Trial({"i": 4}, 3.0, 2e-4)]
    assert at.select(trials, 1e-3).options == {"i": 2}          # i=1 too inaccurate, i=3 failed, tie -> earlier
    assert at.select(trials, 1e-2).options == {"i": 1}
    with pytest.raises(ValueError):
        at.select([at.Trial({}, 1.0, 1.0)], 1e-3)


def test_tune_measures_every_candidate_and_records_failures():
    ref = {"dL_dE": [1.0, 2.0, 2.0]}  # norm 3
    table = {32: (4.0, [1.0, 2.0, 2.0], 40), 64: (2.0, [1.0, 2.0, 2.0015], 31), 128: (1.0, [1.0, 2.3, 2.0], 20)}
    calls = []

    def measure(opts):
        calls.append(opts["restart"])
        if opts["restart"] == 96:
            raise RuntimeError("ncpadj NOT_CONVERGED")
        ms, g, it = table[opts["restart"]]
        return ms, {"dL_dE": g}, it

    cands = [{"restart": m} for m in (32, 64, 96, 128)]
    ch = at.tune(measure, cands, ref, max_rel_err=1e-3)
    assert calls == [32, 64, 96, 128]
    assert ch.options == {"restart": 64} and ch.ms == 2.0 and math.isclose(ch.rel_err, 0.0005, rel_tol=1e-9)
    failed = [t for t in ch.trials if t.error]
    assert len(failed) == 1 and failed[0].options == {"restart": 96} and "NOT_CONVERGED" in failed[0].error
    assert [t.iterations for t in ch.trials if not t.error] == [40, 31, 20]


def test_signature_rounds_sizes_to_powers_of_two():
    assert at.signature(4961, 20000, 451) == "v8192-t32768-c512-s1"
    assert at.signature(4961, 20000, 451) == at.signature(5000, 17000, 300)
    assert at.signature(100, 320, 0, 4) == "v128-t512-c0-s4"


def test_cache_round_trip(tmp_path):
    path = str(tmp_path / "tune.json")
    c = at.Cache(path)
    assert c.get("k") is None
    c.put("k", at.Choice({"precision": "mixed", "restart": 64}, 6.2, 5.9e-5))
    again = at.Cache(path)
    assert again.get("k") == {"precision": "mixed", "restart": 64}
