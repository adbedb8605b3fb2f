"""The co-rotational and ARAP models (App. B.2) on the GPU against the FP64 oracle: adjoint parity
of every gradient, the forward step's converged state, a mesh that mixes all three models tet
by tet, mixed precision, and the reset to Neo-Hookean."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from tests._cases import rel, step_case  # noqa: E402
from tests.test_gpu_parity import KEYS, T, gpu_contacts  # noqa: E402

pytestmark = pytest.mark.gpu

NAMES = ("neo_hookean", "corotational", "arap")


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


def _model(which):
    """The oracle's model argument: a name, or for "mixed" one name per tet of the cube (hashable)."""
    if which != "mixed":
        return which
    nt = synth.cube_drop().scene.tets.shape[0]
    return tuple(NAMES[i % 3] for i in range(nt))


def _scene(pkg, ctx, sc, model):
    s = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    s.set_model(list(model) if isinstance(model, tuple) else model)
    return s


def _adjoint(pkg, scene, case, rtol, seed=0, **kw):
    pb, st, s, q_prev, v_prev = case
    rng = np.random.default_rng(seed)
    dq = 2 * (s.q - pb.q_target) + rng.normal(size=s.q.shape) * 1e-4
    dv = rng.normal(size=s.q.shape) * 1e-3
    ref = st.adjoint(s, q_prev, dq, dv)
    lam = s.lam_frame(st, q_prev) if st.nc else np.zeros((0, 3))
    g, stats = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct), T(s.q), T(q_prev), T(lam), T(dq), T(dv),
                                eps=pb.scene.eps, rtol=rtol, **kw)
    torch.cuda.synchronize()
    errs = {}
    for k, rk in KEYS:
        if st.nc == 0 and k in ("dL_dmu", "dL_dmu_contact"):
            continue
        errs[k] = rel(g[k].cpu().numpy().reshape(-1), np.asarray(ref[rk]).reshape(-1))
    return g, ref, stats, errs


@pytest.mark.parametrize("which", ["corotational", "arap", "mixed"])
@pytest.mark.parametrize("k", [2, 5])
def test_adjoint_parity(pkg, ctx, which, k):
    model = _model(which)
    case = step_case("cube_drop", k, model)
    scene = _scene(pkg, ctx, case[0].scene, model)
    _, _, stats, errs = _adjoint(pkg, scene, case, rtol=1e-12)
    assert stats["rel_residual"] <= 1e-12
    assert max(errs.values()) <= 1e-8, errs


@pytest.mark.parametrize("which", ["corotational", "arap"])
def test_adjoint_mixed_precision(pkg, ctx, which):
    case = step_case("cube_drop", 5, which)
    scene = _scene(pkg, ctx, case[0].scene, which)
    _, _, _, errs = _adjoint(pkg, scene, case, rtol=1e-8, precision="mixed", cap_precision="mixed")
    assert max(errs.values()) <= 1e-3, errs


def test_arap_has_no_lambda_gradient_path(pkg, ctx):
    """ARAP ignores lambda, so E and nu act only through mu = E / (2 (1 + nu)): per tet
    dL/dnu / dL/dE = (dmu/dnu) / (dmu/dE) = -E / (1 + nu)."""
    case = step_case("cube_drop", 2, "arap")
    sc = case[0].scene
    g, _, _, _ = _adjoint(pkg, _scene(pkg, ctx, sc, "arap"), case, rtol=1e-12)
    dE = g["dL_dE"].cpu().numpy()
    dnu = g["dL_dnu"].cpu().numpy()
    expect = -dE * sc.E / (1.0 + sc.nu)
    assert np.allclose(dnu, expect, rtol=1e-10, atol=1e-12 * np.abs(expect).max())


@pytest.mark.parametrize("which", ["corotational", "arap", "mixed"])
def test_forward_matches_oracle_state(pkg, ctx, which):
    model = _model(which)
    pb, st, s, q_prev, v_prev = step_case("cube_drop", 5, model)
    sc = pb.scene
    scene = _scene(pkg, ctx, sc, model)
    # ARAP is not convex under compression: the residual line search damps Newton to t = 1/8 for
    # about 70 iterations before the quadratic phase (the oracle's own Newton takes 89), so the
    # forward gets the oracle's iteration budget
    q, lam, stats = pkg.forward_step(scene, gpu_contacts(pkg, st.ct), T(q_prev), T(v_prev), None,
                                     tuple(sc.gravity), eps=sc.eps, newton_tol=1e-11, max_newton=200)
    assert stats["residual"] < 1e-8
    assert rel(q.cpu().numpy() - q_prev, s.q - q_prev) < 1e-7
    if st.nc:
        assert rel(lam.cpu().numpy(), s.lam_frame(st, q_prev)) < 1e-6


def test_reset_to_neo_hookean_and_invalid_codes(pkg, ctx):
    case = step_case("cube_drop", 2)
    sc = case[0].scene
    scene = _scene(pkg, ctx, sc, "arap")
    scene.set_model("neo_hookean")
    _, _, _, errs = _adjoint(pkg, scene, case, rtol=1e-12)
    assert max(errs.values()) <= 1e-8, errs
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        scene.set_model([3] * scene.n_tets)
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        scene.set_model([-1] + [0] * (scene.n_tets - 1))
