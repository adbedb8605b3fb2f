"""Host logic of two bench legs (CPU only), with fakes for the device parts: the constitutive-model
and bindings timings, and the CPU baseline at the bench's state with its fallbacks."""
import types

import numpy as np
import torch

import bench


class FakeScene:
    def __init__(self, fail_on=None):
        self.models = []
        self.fail_on = fail_on

    def set_model(self, name):
        self.models.append(name)


def _pkg():
    def Bindings(vertex, target, compliance, tet=None, bary=None):
        return types.SimpleNamespace(vertex=vertex, target=target, compliance=compliance)
    return types.SimpleNamespace(Bindings=Bindings)


def test_models_leg_times_each_model_and_the_bindings():
    scene = FakeScene()
    seen = []

    def timed(**kw):
        seen.append((scene.models[-1], kw))
        return 20.0, [{"iterations": 30, "ms_assemble": 0.2}, {"iterations": 32, "ms_assemble": 0.3}]

    q = torch.arange(3 * 4961, dtype=torch.float64).reshape(4961, 3)
    res = bench.models_leg(_pkg(), torch, torch.device("cpu"), scene, 4961, q, timed)
    assert set(res) == {"corotational", "arap", "bindings"}
    assert res["arap"]["gradients_per_s"] == 100.0 and res["arap"]["krylov_iterations"] == 31
    b = seen[-1][1]["bindings"]
    assert seen[-1][0] == "neo_hookean" and res["bindings"]["n"] == 40 == b.vertex.numel()
    assert torch.equal(b.target, q[b.vertex.long()]) and torch.all(b.compliance == 1e-6)
    assert b.vertex.dtype == torch.int32 and len(set(b.vertex.tolist())) == 40
    assert scene.models == ["corotational", "arap", "neo_hookean", "neo_hookean"]


def test_models_leg_reports_a_failure_and_resets_the_model():
    scene = FakeScene()

    def timed(**kw):
        if scene.models[-1] == "arap":
            raise RuntimeError("ncpadj NOT_CONVERGED: Krylov stopped")
        return 10.0, [{"iterations": 30, "ms_assemble": 0.2}]

    res = bench.models_leg(_pkg(), torch, torch.device("cpu"), scene, 100, torch.zeros(100, 3), timed)
    assert "corotational" in res and "arap" not in res and "NOT_CONVERGED" in res["error"]
    assert scene.models[-1] == "neo_hookean"


def _arrays():
    return {"q": np.zeros((4, 3)), "q_prev": np.zeros((4, 3)), "dL_dq": np.ones((4, 3)), "dL_dv": np.zeros((4, 3)),
            "fp64/z": np.ones((4, 3))}


def test_cpu_baseline_at_the_bench_state(monkeypatch):
    calls = []

    def fake(steps, warmup, state=None, batch=False):
        calls.append(state)
        d = np.load(state)
        assert sorted(d.files) == sorted(_arrays())
        return {"seconds": [2.0, 2.0, 2.0], "threads": 1, "rel_err_vs_oracle": {"fp64": 1e-9}}

    monkeypatch.setattr(bench, "oracle_times", fake)
    cpu, err = bench.cpu_baseline_leg(_arrays())
    assert cpu["value"] == 0.5 and cpu["cores"] == 1 and "GPU state" in cpu["sample"] and err == {"fp64": 1e-9}
    assert len(calls) == 1 and calls[0] is not None


def test_cpu_baseline_falls_back_to_the_start_point(monkeypatch):
    def fake(steps, warmup, state=None, batch=False):
        if state is not None:
            raise RuntimeError("the given state is outside the local contact solve's domain")
        return {"seconds": [1.0, 1.0], "threads": 1}

    monkeypatch.setattr(bench, "oracle_times", fake)
    cpu, err = bench.cpu_baseline_leg(_arrays())
    assert cpu["value"] == 1.0 and "start point" in cpu["sample"] and err is None


def test_cpu_baseline_reports_a_double_failure(monkeypatch):
    def fake(steps, warmup, state=None, batch=False):
        raise RuntimeError("oracle failed")

    monkeypatch.setattr(bench, "oracle_times", fake)
    cpu, err = bench.cpu_baseline_leg(_arrays())
    assert cpu["value"] is None and "failed" in cpu["sample"] and err is None


def test_cpu_baseline_of_the_batch_names_its_sample(monkeypatch):
    def fake(steps, warmup, state=None, batch=False):
        assert batch and state is not None
        return {"seconds": [1.0, 3.0], "threads": 1, "blocks": [{"block": 4}, {"block": 9}],
                "rel_err_vs_oracle": {"mixed": 2e-5}}

    monkeypatch.setattr(bench, "oracle_times", fake)
    cpu, err = bench.cpu_baseline_leg({"b4/q": np.zeros((2, 3))}, batch=True)
    assert cpu["value"] == 0.5 and "[4, 9]" in cpu["sample"] and "seeded sample" in cpu["sample"]
    assert err == {"mixed": 2e-5}


def test_krylov_summary_counts_the_blocks_own_iterations():
    sts = [[{"iterations": 5}, {"iterations": 7}], [{"iterations": 10}, {"iterations": 30}, {"iterations": 0}]]
    assert bench.krylov_summary(sts) == {"per_block_sum": 40, "per_block_max": 30, "per_block_mean": 40 / 3,
                                         "blocks_x_max": 90}


def test_profiled_traffic_is_dropped_once_the_kernels_change(tmp_path, monkeypatch):
    """The traffic of the committed capture stands while the two kernels' source text is unchanged,
    whatever else changes in their file."""
    src = open(bench.os.path.join(bench.ROOT, "paper_2603_16478_gb300", "csrc", "linalg.cu")).read()
    digest = bench.spmv_kernels_digest(src)
    assert digest is not None
    assert bench.spmv_kernels_digest(src + "\n// another kernel\n") == digest
    edited = src.replace("a0 = warp_sum(a0);", "a0 = warp_sum(a0) * 1;", 1)
    assert bench.spmv_kernels_digest(edited) != digest
    prof = tmp_path / "p.md"
    monkeypatch.setattr(bench, "TRAFFIC_PROFILE", str(prof))
    assert bench.profiled_traffic()[0] is None
    prof.write_text(f"traffic_bytes_per_apply: 1234\nspmv_kernels_sha256: {digest}\n")
    assert bench.profiled_traffic()[0] == 1234
    prof.write_text("traffic_bytes_per_apply: 1234\nspmv_kernels_sha256: " + "0" * 64 + "\n")
    assert bench.profiled_traffic() == (None, "kernels changed since the ncu capture")


def test_clock_sampler_parses_nvidia_smi_lines():
    """Median SM clock, maximum clock and the throttle reasons seen active in any sample."""
    cs = bench.ClockSampler(0)
    cs.proc = types.SimpleNamespace(terminate=lambda: None, wait=lambda timeout=None: 0, kill=lambda: None)
    cs.lines = ["0, 2070, 2070, 700.5, 0x0, Not Active, Not Active, Not Active, Not Active",
                "0, 1980, 2070, 1399.0, 0x4, Not Active, Not Active, Not Active, Active",
                "0, 2070, 2070, 900.0, 0x0, Not Active, Not Active, Not Active, Not Active",
                "garbage line", "0, [N/A], 2070, 1.0, 0x0, Not Active, Not Active, Not Active, Not Active"]
    out = cs.stop()
    assert out == {"sm_mhz": 2070.0, "sm_max_mhz": 2070.0, "reasons": ["sw_power_cap"], "samples": 3}
    none = bench.ClockSampler(0)
    assert none.stop()["reasons"] == ["nvidia-smi unavailable"]
