"""Per-tet actuation (constant active stress a_i d_i d_i^T along a fibre d_i): the GPU forward
step with activations and the adjoint's dL/da against the oracle."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from oracle.actuation import actuation_force, actuation_gradient  # noqa: E402
from tests._cases import rel, step_case  # noqa: E402
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


@pytest.mark.parametrize("k", [2, 5])
def test_actuated_step_and_activation_gradient(pkg, ctx, k):
    pb, st, base, q_prev, v_prev = step_case("cube_drop", k)
    sc = pb.scene
    act, fibre = synth.random_actuation(st.mesh.n_tets, seed=k)
    ref = st.forward(q_prev, v_prev, f_ctrl=actuation_force(st.mesh, act.astype(float), fibre), q_init=base.q)
    assert ref.residual < 1e-8
    g_ref = st.adjoint(ref, q_prev, 2 * (ref.q - pb.q_target), np.zeros_like(q_prev))
    da_ref = actuation_gradient(st.mesh, g_ref["z"], fibre, sc.h)

    scene = gpu_scene(pkg, ctx, sc)
    scene.set_fibres(fibre)
    c = gpu_contacts(pkg, st.ct)
    a_dev = torch.tensor(act, device="cuda")
    # the activations push the lightest vertices at ~300 m/s^2: the inertial prediction inverts tets
    # and the solve starts from a point pulled back towards q_prev
    q, lam, stats = pkg.forward_step(scene, c, T(q_prev), T(v_prev), None, tuple(sc.gravity), eps=sc.eps,
                                     newton_tol=1e-11, max_newton=300, act=a_dev)
    assert stats["residual"] < 1e-8
    # a sticking contact (slip ~1e-7) has two converged solutions, slip and gamma both flipped (the
    # same force): the GPU state must be one of the oracle's, from base.q or from its own start
    own = st.forward(q_prev, v_prev, f_ctrl=actuation_force(st.mesh, act.astype(float), fibre))
    dq = q.cpu().numpy() - q_prev
    assert min(rel(dq, ref.q - q_prev), rel(dq, own.q - q_prev)) < 1e-7
    # adjoint at the oracle's state, so that dL/da is compared on identical inputs
    lam_ref = T(ref.lam_frame(st, q_prev)) if st.nc else None
    g, stats = pkg.adjoint_step(scene, c, T(ref.q), T(q_prev), lam_ref, T(2 * (ref.q - pb.q_target)), None,
                                eps=sc.eps, want=("dL_dact", "dL_dfext", "z"))
    assert g["dL_dact"].dtype == torch.float32
    assert rel(g["dL_dact"].cpu().numpy(), da_ref) < 1e-6
    # same numbers through host memory
    gh, _ = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct, "cpu"), T(ref.q, dev="cpu"), T(q_prev, dev="cpu"),
                             None if lam_ref is None else lam_ref.cpu(), T(2 * (ref.q - pb.q_target), dev="cpu"),
                             None, eps=sc.eps, memory="host", want=("dL_dact",))
    assert rel(gh["dL_dact"].numpy(), da_ref) < 1e-6


def test_actuation_requires_fibres(pkg, ctx):
    pb, st, base, q_prev, v_prev = step_case("cube_drop", 2)
    sc = pb.scene
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)  # no fibres set
    a_dev = torch.zeros(st.mesh.n_tets, dtype=torch.float32, device="cuda")
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        pkg.forward_step(scene, gpu_contacts(pkg, st.ct), T(q_prev), T(v_prev), None, tuple(sc.gravity),
                         eps=sc.eps, act=a_dev)
    bad = np.ones((st.mesh.n_tets, 3))
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        scene.set_fibres(bad)
