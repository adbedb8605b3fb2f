"""BiCGSTAB as the Krylov method (NCPADJ_SOLVER_BICGSTAB) against the FP64 oracle, and against
GMRES on the full-size beam."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import rel, step_case  # noqa: E402
from tests.test_gpu_parity import T, assert_parity, gpu_contacts, gpu_scene, run_both  # noqa: E402

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


@pytest.mark.parametrize("name,k", [("cube_drop", 2), ("cube_drop", 5), ("two_tet", 1)])
@pytest.mark.parametrize("precond", ["woodbury", "jacobi"])
def test_bicgstab_parity(pkg, ctx, name, k, precond):
    case = step_case(name, k)
    g, ref, stats = run_both(pkg, ctx, case, rtol=1e-12, solver="bicgstab", precond=precond, max_iters=5000)
    assert stats["solver_used"] == 3 and stats["rel_residual"] <= 1e-12
    assert_parity(g, ref, 1e-8, case[1].nc)


def test_bicgstab_mixed_precision(pkg, ctx):
    case = step_case("cube_drop", 5)
    g, ref, stats = run_both(pkg, ctx, case, rtol=1e-6, solver="bicgstab", precision="mixed")
    assert stats["solver_used"] == 3
    assert_parity(g, ref, 1e-3, case[1].nc)


def test_bicgstab_matches_gmres_on_the_beam(pkg, ctx):
    import synth
    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    scene = gpu_scene(pkg, ctx, sc)
    c = gpu_contacts(pkg, ct)
    q_prev, v_prev = T(pb.q0), T(pb.v0)
    q, lam, _ = pkg.forward_step(scene, c, q_prev, v_prev, None, tuple(sc.gravity), eps=sc.eps)
    dq = T(np.random.default_rng(2).normal(size=pb.q0.shape))
    gg, sg = pkg.adjoint_step(scene, c, q, q_prev, lam.contiguous(), dq, None, eps=sc.eps, rtol=1e-10)
    gb, sb = pkg.adjoint_step(scene, c, q, q_prev, lam.contiguous(), dq, None, eps=sc.eps, rtol=1e-10,
                              solver="bicgstab", max_iters=5000)
    torch.cuda.synchronize()
    assert sb["solver_used"] == 3 and sb["rel_residual"] <= 1e-10
    for key in ("z", "dL_dq_prev", "dL_dE", "dL_dmu"):
        assert rel(gb[key].cpu().numpy(), gg[key].cpu().numpy()) <= 1e-6, key
