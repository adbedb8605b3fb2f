"""The GPU forward step (which produces the converged states the adjoint needs) reaches the
oracle's converged state."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import rel, rollout, step_case  # noqa: E402
from tests.test_gpu_parity import T, gpu_contacts, gpu_scene  # noqa: E402

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


@pytest.mark.parametrize("name,k", [("cube_drop", 1), ("cube_drop", 2), ("cube_drop", 5), ("two_tet", 1)])
def test_forward_matches_oracle_state(pkg, ctx, name, k):
    pb, st, s, q_prev, v_prev = step_case(name, k)
    sc = pb.scene
    scene = gpu_scene(pkg, ctx, sc)
    q, lam, stats = pkg.forward_step(scene, gpu_contacts(pkg, st.ct), T(q_prev), T(v_prev), None,
                                     tuple(sc.gravity), eps=sc.eps, newton_tol=1e-11)
    assert stats["residual"] < 1e-8
    dq_ref = s.q - q_prev
    assert rel(q.cpu().numpy() - q_prev, dq_ref) < 1e-7
    if st.nc:
        assert rel(lam.cpu().numpy(), s.lam_frame(st, q_prev)) < 1e-6


def test_forward_then_adjoint_on_gpu_state(pkg, ctx):
    """A GPU-forward state is a valid input for the adjoint (converges, finite gradients)."""
    pb, q_prev, v_prev = rollout("cube_drop", 4)
    sc = pb.scene
    ct = sc.contacts(q_prev)
    scene = gpu_scene(pkg, ctx, sc)
    c = gpu_contacts(pkg, ct)
    q, lam, _ = pkg.forward_step(scene, c, T(q_prev), T(v_prev), None, tuple(sc.gravity), eps=sc.eps)
    g, stats = pkg.adjoint_step(scene, c, q, T(q_prev), lam.contiguous(), 2 * (q - T(pb.q_target)), None, eps=sc.eps)
    assert stats["rel_residual"] <= 1e-8
    assert torch.isfinite(g["dL_dE"]).all()
