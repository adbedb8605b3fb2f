"""ncpadj_scene_refactor: a scene given a new material (E, nu) computes what a scene built with that
material computes -- the adjoint against the oracle's at the new material, and the forward state --
and a rejected material leaves the scene as it was."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import make_step, rel, rollout  # noqa: E402
from tests.test_gpu_parity import T, assert_parity, gpu_contacts  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_refactored_scene_matches_the_oracle_at_the_new_material(pkg, precision):
    ctx = pkg.Context(0)
    pb, q_prev, v_prev = rollout("cube_drop", 4)
    sc = pb.scene
    rng = np.random.default_rng(5)
    E1 = sc.E * rng.uniform(1.2, 1.8, sc.E.shape)  # per tet
    nu1 = np.full_like(sc.nu, 0.35)
    st = make_step(sc, sc.contacts(q_prev), E=E1, nu=nu1)
    s = st.forward(q_prev, v_prev)
    assert s.residual < 1e-8
    dq = 2 * (s.q - pb.q_target) + rng.normal(size=s.q.shape) * 1e-4
    dv = rng.normal(size=s.q.shape) * 1e-3
    ref = st.adjoint(s, q_prev, dq, dv)
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)  # built for the old material
    scene.refactor(E1, nu1)
    E, nu = scene.material()
    assert np.array_equal(E.numpy(), E1) and np.array_equal(nu.numpy(), nu1)
    g, _ = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct), T(s.q), T(q_prev), T(s.lam_frame(st, q_prev)), T(dq),
                            T(dv), eps=sc.eps, rtol=1e-12 if precision == "fp64" else 1e-8, precision=precision,
                            cap_precision=precision)
    torch.cuda.synchronize()
    assert_parity(g, ref, 1e-8 if precision == "fp64" else 1e-3, st.nc)
    if precision == "fp64":  # the forward on the refactored scene reaches the oracle's state
        q, _, fs = pkg.forward_step(scene, gpu_contacts(pkg, st.ct), T(q_prev), T(v_prev), None, tuple(sc.gravity),
                                    eps=sc.eps, newton_tol=1e-11)
        assert rel(q.cpu().numpy() - q_prev, s.q - q_prev) < 1e-7


def test_a_rejected_material_leaves_the_scene_unchanged(pkg):
    ctx = pkg.Context(0)
    pb, q_prev, v_prev = rollout("cube_drop", 4)
    sc = pb.scene
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    x = torch.randn(sc.X.shape[0], 3, dtype=torch.float64, device="cuda")
    y0 = pkg.elastic_solve(scene, x).clone()
    bad_E = sc.E.copy()
    bad_E[7] = -1.0
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        scene.refactor(bad_E, sc.nu)
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        scene.refactor(sc.E, np.full_like(sc.nu, 0.5))
    E, nu = scene.material()
    assert np.array_equal(E.numpy(), sc.E) and np.array_equal(nu.numpy(), sc.nu)
    assert torch.equal(pkg.elastic_solve(scene, x), y0)
