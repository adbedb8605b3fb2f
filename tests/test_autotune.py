"""Host-side logic of the adjoint autotuner (CPU only): candidate grid, accuracy-gated selection,
failure handling, signatures and the persistent cache.  The timed calls are faked."""
import math

import pytest

from paper_2603_16478_gb300 import autotune as at


def test_default_candidates_cover_every_variant_and_restart():
    c = at.default_candidates(451)
    assert len(c) == 5 * 3
    assert {(x["precision"], x["cap_precision"]) for x in c} == set(at.PRECISION_VARIANTS)
    assert {x["restart"] for x in c} == {32, 64, 128} and {x["cap_block"] for x in c} == {0}
    big = at.default_candidates(2329)
    assert len(big) == 5 * 3 * 2 and {x["cap_block"] for x in big} == {0, 1024}


def test_tune_shape_times_every_shape_and_applies_the_fastest():
    applied, cost = [], {128: 3.0, 256: 2.0, 512: 2.5, 1024: None}

    def apply(sh):
        applied.append(sh)

    def measure():
        c = cost[applied[-1]]
        if c is None:
            raise RuntimeError("INVALID_ARG")
        return c

    best, times = at.tune_shape(apply, measure, [128, 256, 512, 1024])
    assert best == 256 and applied[-1] == 256
    assert times[128] == 3.0 and times[512] == 2.5 and math.isinf(times[1024])
    with pytest.raises(ValueError):
        at.tune_shape(apply, lambda: (_ for _ in ()).throw(RuntimeError("x")), [128])


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


def test_tune_adjoint_glue_with_fake_device(monkeypatch, tmp_path):
    """tune_adjoint end to end with a fake adjoint call and fake CUDA events: the FP64 reference,
    per-candidate timing (median of the repeats), the accuracy gate, the choice and the cache."""
    import contextlib
    import types

    import torch

    from paper_2603_16478_gb300 import binding

    clock = {"t": 0.0, "calls": 0}
    base = {("fp64", "fp64"): 10.0, ("mixed", "fp64"): 8.0, ("mixed", "mixed"): 5.0, ("mixed", "tf32x3"): 4.0,
            ("mixed", "refined"): 4.5}
    err = {("fp64", "fp64"): 0.0, ("mixed", "fp64"): 5e-5, ("mixed", "mixed"): 2e-3, ("mixed", "tf32x3"): 5e-4,
           ("mixed", "refined"): 5e-5}
    chunk_cost = {128: 1.0, 256: 0.0, 512: -0.25}

    def fake_adjoint(scene, contacts, q, q_prev, lam, dL_dq, dL_dv, *, precision, cap_precision, restart,
                     cap_block, **kw):
        clock["calls"] += 1
        clock["t"] += base[(precision, cap_precision)] + chunk_cost[scene.chunk] - (0.5 if restart == 128 else 0.0)
        e = err[(precision, cap_precision)]
        g = {"dL_dq_prev": torch.ones(4, 3, dtype=torch.float64) * (1 + e), "dL_dE": torch.ones(6, dtype=torch.float64)}
        return g, {"iterations": 30}

    class FakeEvent:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock["t"]

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(binding, "adjoint_step", fake_adjoint)
    monkeypatch.setattr(torch.cuda, "Stream", lambda dev=None: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda dev=None: None)
    scene = types.SimpleNamespace(n_verts=4961, n_tets=20000, info=lambda: {"n_scenes": 1}, chunk=256)
    scene.set_chunk = lambda n: setattr(scene, "chunk", int(n))
    contacts = types.SimpleNamespace(n=451)
    q = torch.zeros(4, 3, dtype=torch.float64)
    cache = at.Cache(str(tmp_path / "tune.json"))
    ch = at.tune_adjoint(scene, contacts, q, q, q, q, None, repeats=3, cache=cache)
    # launch shape first (timed with the tensor-core variant), then the options at that shape
    assert ch.chunk == 512 and scene.chunk == 512 and ch.chunk_ms == {128: 5.0, 256: 4.0, 512: 3.75}
    assert ch.options == {"precision": "mixed", "cap_precision": "tf32x3", "restart": 128, "cap_block": 0}
    assert ch.ms == 3.25 and abs(ch.rel_err - 5e-4) < 1e-12
    assert len(ch.trials) == 15 and clock["calls"] == 1 + 3 * (1 + 3) + 15 * (1 + 3)
    calls = clock["calls"]
    scene.chunk = 256
    again = at.tune_adjoint(scene, contacts, q, q, q, q, None, cache=at.Cache(str(tmp_path / "tune.json")))
    assert again.options == ch.options and clock["calls"] == calls  # from the cache, nothing run
    assert again.chunk == 512 and scene.chunk == 512                # the cached shape is applied


def test_tune_adjoint_shape_stage_falls_back_to_fp64_and_keeps_the_chunk(monkeypatch):
    """Where the tensor-core variant fails on a scene the launch shape is timed with plain FP64; where
    nothing runs the scene keeps its chunk length and the option stage still reports the failures."""
    import contextlib
    import types

    import torch

    from paper_2603_16478_gb300 import binding

    clock = {"t": 0.0}
    broken = {("mixed", "tf32x3")}
    cost = {128: 3.0, 256: 2.0, 512: 2.5}

    def fake_adjoint(scene, contacts, q, q_prev, lam, dL_dq, dL_dv, *, precision, cap_precision, restart,
                     cap_block, **kw):
        if (precision, cap_precision) in broken or scene.dead:
            raise RuntimeError("ncpadj NOT_CONVERGED")
        clock["t"] += cost[scene.chunk]
        return {"dL_dE": torch.ones(3, dtype=torch.float64)}, {"iterations": 10}

    class FakeEvent:
        def __init__(self, enable_timing=False):
            self.t = None

        def record(self, stream=None):
            self.t = clock["t"]

        def synchronize(self):
            pass

        def elapsed_time(self, other):
            return other.t - self.t

    monkeypatch.setattr(binding, "adjoint_step", fake_adjoint)
    monkeypatch.setattr(torch.cuda, "Stream", lambda dev=None: types.SimpleNamespace(cuda_stream=0))
    monkeypatch.setattr(torch.cuda, "stream", lambda s: contextlib.nullcontext())
    monkeypatch.setattr(torch.cuda, "Event", FakeEvent)
    monkeypatch.setattr(torch.cuda, "synchronize", lambda dev=None: None)
    scene = types.SimpleNamespace(n_verts=10, n_tets=20, info=lambda: {"n_scenes": 1}, chunk=512, dead=False)
    scene.set_chunk = lambda n: setattr(scene, "chunk", int(n))
    q = torch.zeros(2, 3, dtype=torch.float64)
    cands = [{"precision": "fp64", "cap_precision": "fp64", "restart": 64, "cap_block": 0}]
    ch = at.tune_adjoint(scene, types.SimpleNamespace(n=0), q, q, q, q, None, candidates=cands, repeats=1)
    assert ch.chunk == 256 and scene.chunk == 256 and ch.chunk_ms == {128: 3.0, 256: 2.0, 512: 2.5}
    # nothing runs at all: the reference call itself fails before any stage
    scene.dead, scene.chunk = True, 512
    with pytest.raises(RuntimeError):
        at.tune_adjoint(scene, types.SimpleNamespace(n=0), q, q, q, q, None, candidates=cands, repeats=1)
    assert scene.chunk == 512
