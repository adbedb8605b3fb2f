"""Mixed precision (FP32 matrix values, SVD Jacobians, matvec and preconditioner apply; FP64
vectors, dot products, Gram-Schmidt and Hessenberg) against the FP64 oracle and the GPU FP64
path.  The target is <= 1e-3 relative error per gradient block."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import rel, step_case  # noqa: E402
from tests.test_gpu_parity import KEYS, T, gpu_contacts, gpu_scene, run_both  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    return pkg.Context(0)


def _errors(g, ref, nc):
    out = {}
    for k, rk in KEYS:
        if nc == 0 and k in ("dL_dmu", "dL_dmu_contact"):
            continue
        out[k] = rel(g[k].cpu().numpy().reshape(-1), np.asarray(ref[rk]).reshape(-1))
    return out


@pytest.mark.parametrize("cap", ["fp64", "mixed", "tf32x3", "refined"])
@pytest.mark.parametrize("name,k", [("cube_drop", 0), ("cube_drop", 2), ("cube_drop", 5), ("two_tet", 1)])
def test_mixed_against_oracle(pkg, ctx, name, k, cap):
    case = step_case(name, k)
    g, ref, stats = run_both(pkg, ctx, case, rtol=1e-8, precision="mixed", cap_precision=cap)
    errs = _errors(g, ref, case[1].nc)
    assert max(errs.values()) <= 1e-3, errs


@pytest.mark.parametrize("cap", ["fp64", "mixed", "tf32x3", "refined"])
def test_mixed_against_fp64_on_the_beam(pkg, ctx, cap):
    """Full-size beam (20k tets, 451 contacts): GPU mixed vs GPU FP64 on a GPU-forward state."""
    import synth
    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    scene = gpu_scene(pkg, ctx, sc)
    c = gpu_contacts(pkg, ct)
    q_prev, v_prev = T(pb.q0), T(pb.v0)
    for _ in range(2):
        q, lam, _ = pkg.forward_step(scene, c, q_prev, v_prev, None, tuple(sc.gravity), eps=sc.eps)
        v_prev = (q - q_prev) / sc.h
        q_prev_step, q_prev = q_prev, q
    rng = np.random.default_rng(1)
    dq = T(rng.normal(size=pb.q0.shape))
    g64, s64 = pkg.adjoint_step(scene, c, q, q_prev_step, lam.contiguous(), dq, None, eps=sc.eps)
    g32, s32 = pkg.adjoint_step(scene, c, q, q_prev_step, lam.contiguous(), dq, None, eps=sc.eps, precision="mixed",
                                cap_precision=cap)
    torch.cuda.synchronize()
    for k, _ in KEYS:
        e = rel(g32[k].cpu().numpy(), g64[k].cpu().numpy())
        assert e <= 1e-3, (k, e)


def test_tensor_core_capacitance_keeps_fp64_results_and_iterations(pkg, ctx):
    """The tensor-core capacitance inverse only preconditions: with FP64 matrices the gradients match
    the oracle to 1e-8 at rtol 1e-12, in about as many iterations as the FP32 Gauss-Jordan inverse; the
    refined solve (one refinement step against the FP64 capacitance) is an FP64-accurate capacitance
    solve, so it takes the iterations of the FP64 inverse."""
    from tests.test_gpu_parity import assert_parity
    case = step_case("cube_drop", 5)
    its = {}
    for cap in ("fp64", "mixed", "tf32x3", "refined"):
        g, ref, stats = run_both(pkg, ctx, case, rtol=1e-12, cap_precision=cap)
        assert_parity(g, ref, 1e-8, case[1].nc)
        its[cap] = stats["iterations"]
    assert its["tf32x3"] <= its["mixed"] + 2, its
    assert its["refined"] <= its["fp64"] + 1, its


def test_refined_capacitance_matches_fp64_iterations_on_the_beam(pkg, ctx):
    """Full-size beam (1,353-row capacitance): the refined FP32 tensor-core solve preconditions like the
    FP64 inverse (same GMRES iterations within one) and the gradients agree to the solve tolerance."""
    import synth
    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    scene = gpu_scene(pkg, ctx, sc)
    c = gpu_contacts(pkg, ct)
    q_prev, v_prev = T(pb.q0), T(pb.v0)
    for _ in range(2):
        q, lam, _ = pkg.forward_step(scene, c, q_prev, v_prev, None, tuple(sc.gravity), eps=sc.eps)
        v_prev = (q - q_prev) / sc.h
        q_prev_step, q_prev = q_prev, q
    rng = np.random.default_rng(2)
    dq = T(rng.normal(size=pb.q0.shape))
    out = {}
    for cap in ("fp64", "refined"):
        out[cap] = pkg.adjoint_step(scene, c, q, q_prev_step, lam.contiguous(), dq, None, eps=sc.eps, rtol=1e-10,
                                    cap_precision=cap)
    torch.cuda.synchronize()
    (g64, s64), (gr, sr) = out["fp64"], out["refined"]
    assert sr["iterations"] <= s64["iterations"] + 1, (sr["iterations"], s64["iterations"])
    for k, _ in KEYS:
        e = rel(gr[k].cpu().numpy(), g64[k].cpu().numpy())
        assert e <= 1e-8, (k, e)
