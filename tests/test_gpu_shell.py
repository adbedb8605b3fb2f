"""Shells on the GPU (ncpadj_scene_create_shells, App. B.1's 2D formulation with isometric
bending) against the oracle's triangle elements, element by element: the adjoint gradients of a
cloth draped over a sphere (frictional and frictionless contacts, the three projection models, FP64
and mixed precision, one mesh and a batch), the bending-stiffness gradient, a new bending stiffness,
the forward step, and the argument checks of the shell entry points."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from tests._cases import make_step, rel, step_case  # noqa: E402
from tests.test_gpu_parity import KEYS, T, assert_parity, gpu_contacts  # noqa: E402

pytestmark = pytest.mark.gpu

CLOTH = dict(n=5, size=0.1, radius=0.04, height=0.002, mu=0.3, bend=2e-4, E=3e4)


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


def shell_scene(pkg, ctx, scenes, model="neo_hookean"):
    s = pkg.Scene.shells(ctx, [(sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.thickness, sc.bend) for sc in scenes],
                         scenes[0].h)
    if model != "neo_hookean":
        s.set_model(model)
    return s


def cloth_case(k, model="neo_hookean", **over):
    return step_case("cloth_drape", k, model, **dict(CLOTH, **over))


def seeds(s, pb, seed):
    rng = np.random.default_rng(seed)
    return 2 * (s.q - pb.q_target) + rng.normal(size=s.q.shape) * 1e-4, rng.normal(size=s.q.shape) * 1e-3


def run_shell(pkg, ctx, case, model="neo_hookean", seed=0, rtol=1e-12, scene=None, **kw):
    pb, st, s, q_prev, v_prev = case
    dq, dv = seeds(s, pb, seed)
    ref = st.adjoint(s, q_prev, dq, dv)
    scene = scene or shell_scene(pkg, ctx, [pb.scene], model)
    lam = s.lam_frame(st, q_prev) if st.nc else np.zeros((0, 3))
    want = ("dL_dq_prev", "dL_dv_prev", "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu", "dL_dmu_contact", "z", "dL_dbend")
    g, stats = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct), T(s.q), T(q_prev), T(lam), T(dq), T(dv),
                                eps=pb.scene.eps, rtol=rtol, want=want, **kw)
    torch.cuda.synchronize()
    return g, ref, stats


@pytest.mark.parametrize("k", [0, 3, 5])
def test_cloth_fp64_parity(pkg, ctx, k):
    case = cloth_case(k)
    if k:
        assert case[1].nc > 0
    g, ref, stats = run_shell(pkg, ctx, case)
    assert stats["rel_residual"] <= 1e-12
    assert_parity(g, ref, 1e-8, case[1].nc)
    assert rel(g["dL_dbend"].cpu().numpy(), [ref["dL_dbend"]]) < 1e-8


@pytest.mark.parametrize("model", ["corotational", "arap"])
def test_cloth_models_parity(pkg, ctx, model):
    case = cloth_case(3, model)
    g, ref, stats = run_shell(pkg, ctx, case, model)
    assert_parity(g, ref, 1e-8, case[1].nc)
    assert rel(g["dL_dbend"].cpu().numpy(), [ref["dL_dbend"]]) < 1e-8


def test_frictionless_cloth_uses_cg(pkg, ctx):
    case = cloth_case(3, mu=0.0)
    g, ref, stats = run_shell(pkg, ctx, case)
    assert stats["solver_used"] == 1  # CG
    assert_parity(g, ref, 1e-8, case[1].nc)


def test_cloth_mixed_precision(pkg, ctx):
    """FP32 matrix values (the triangles' Jacobian blocks, bending and contact blocks): the solve is of
    a system rounded to FP32, so each gradient block agrees to ~1e-6 in relative 2-norm (the mixed
    path's target is 1e-3, as for tets); single entries that are sums of cancelling terms carry the
    absolute error of their block, so they are not checked one by one."""
    case = cloth_case(3)
    g, ref, stats = run_shell(pkg, ctx, case, rtol=1e-10, precision="mixed")
    for k, rk in KEYS:
        assert rel(g[k].cpu().numpy().reshape(-1), np.asarray(ref[rk]).reshape(-1)) <= 1e-5, k
    assert rel(g["dL_dbend"].cpu().numpy(), [ref["dL_dbend"]]) < 1e-5


def test_cloth_at_paper_tolerance_with_host_memory(pkg, ctx):
    pb, st, s, q_prev, v_prev = cloth_case(3)
    dq, dv = seeds(s, pb, 1)
    ref = st.adjoint(s, q_prev, dq, dv)
    scene = shell_scene(pkg, ctx, [pb.scene])
    lam = s.lam_frame(st, q_prev)
    g, stats = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct, "cpu"), T(s.q, dev="cpu"), T(q_prev, dev="cpu"),
                                T(lam, dev="cpu"), T(dq, dev="cpu"), T(dv, dev="cpu"), eps=pb.scene.eps, rtol=1e-8,
                                memory="host", want=("dL_dE", "dL_dnu", "dL_dq_prev", "z", "dL_dbend"))
    for k in ("dL_dE", "dL_dnu", "dL_dq_prev", "z"):
        assert rel(g[k].numpy().reshape(-1), np.asarray(ref[k]).reshape(-1)) < 1e-5, k
    assert rel(g["dL_dbend"].numpy(), [ref["dL_dbend"]]) < 1e-5


def test_scene_info_counts_triangles_and_hinges(pkg, ctx):
    pb = synth.cloth_drape(**CLOTH)
    scene = shell_scene(pkg, ctx, [pb.scene])
    info = scene.info()
    st = make_step(pb.scene, pb.scene.contacts(pb.q0))
    assert info["element_verts"] == 3 and info["n_tets"] == len(pb.scene.tets)
    assert info["n_hinges"] == len(st.mesh.bending_stencils())
    assert float(scene.bending()[0]) == CLOTH["bend"]


def test_new_bending_stiffness(pkg, ctx):
    """ncpadj_scene_set_bending rebuilds A_s and its factor: the adjoint with k_b' matches the oracle
    step built with k_b'."""
    pb, st, s, q_prev, v_prev = cloth_case(3)
    scene = shell_scene(pkg, ctx, [pb.scene])
    kb = 5 * CLOTH["bend"]
    scene.set_bending(kb)
    assert float(scene.bending()[0]) == kb
    st2 = make_step(pb.scene, st.ct, bend=kb)
    s2 = st2.forward(q_prev, v_prev, q_init=s.q)
    g, ref, _ = run_shell(pkg, ctx, (pb, st2, s2, q_prev, v_prev), scene=scene)
    assert_parity(g, ref, 1e-8, st2.nc)
    assert rel(g["dL_dbend"].cpu().numpy(), [ref["dL_dbend"]]) < 1e-8


def test_cloth_batch_matches_each_mesh(pkg, ctx):
    """Three cloths of different stiffness and bending in one batch call: every mesh's gradients
    equal the oracle's for that mesh alone."""
    cases = [cloth_case(3, E=E, bend=kb) for E, kb in ((3e4, 2e-4), (1e5, 5e-5), (2e4, 1e-3))]
    scene = shell_scene(pkg, ctx, [c[0].scene for c in cases])
    refs, args = [], {k: [] for k in ("ct", "q", "qp", "lam", "dq", "dv")}
    for i, (pb, st, s, q_prev, v_prev) in enumerate(cases):
        dq, dv = seeds(s, pb, 10 + i)
        refs.append(st.adjoint(s, q_prev, dq, dv))
        args["ct"].append(gpu_contacts(pkg, st.ct))
        args["q"].append(T(s.q))
        args["qp"].append(T(q_prev))
        args["lam"].append(T(s.lam_frame(st, q_prev) if st.nc else np.zeros((0, 3))))
        args["dq"].append(T(dq))
        args["dv"].append(T(dv))
    outs, stats = pkg.adjoint_batch(scene, args["ct"], args["q"], args["qp"], args["lam"], args["dq"], args["dv"],
                                    eps=cases[0][0].scene.eps, rtol=1e-12,
                                    want=tuple(k for k, _ in KEYS) + ("dL_dbend",))
    torch.cuda.synchronize()
    for (pb, st, *_), g, ref in zip(cases, outs, refs):
        assert_parity(g, ref, 1e-8, st.nc)
        assert rel(g["dL_dbend"].cpu().numpy(), [ref["dL_dbend"]]) < 1e-8


@pytest.mark.parametrize("k", [1, 3])
def test_cloth_forward_matches_the_oracle(pkg, ctx, k):
    pb, st, s, q_prev, v_prev = cloth_case(k)
    sc = pb.scene
    scene = shell_scene(pkg, ctx, [sc])
    q, lam, stats = pkg.forward_step(scene, gpu_contacts(pkg, st.ct), T(q_prev), T(v_prev), None, tuple(sc.gravity),
                                     eps=sc.eps, newton_tol=1e-11)
    assert stats["residual"] < 1e-8
    assert rel(q.cpu().numpy() - q_prev, s.q - q_prev) < 1e-7
    if st.nc:
        assert rel(lam.cpu().numpy(), s.lam_frame(st, q_prev)) < 1e-6


def test_shell_arguments_are_checked(pkg, ctx):
    X, tris = synth.tri_grid(2, 2, 0.1, 0.1)
    E, nu = np.full(len(tris), 1e5), np.full(len(tris), 0.3)
    good = (X, tris, E, nu, 1000.0, 1e-3, 1e-4)
    with pytest.raises(pkg.NcpadjError, match="thickness"):
        pkg.Scene.shells(ctx, [(X, tris, E, nu, 1000.0, 0.0, 1e-4)], 0.01)
    with pytest.raises(pkg.NcpadjError, match="bend"):
        pkg.Scene.shells(ctx, [(X, tris, E, nu, 1000.0, 1e-3, -1.0)], 0.01)
    bad = tris.copy()
    bad[0, 2] = bad[0, 1]  # a collapsed triangle
    with pytest.raises(pkg.NcpadjError, match="degenerate"):
        pkg.Scene.shells(ctx, [(X, bad, E, nu, 1000.0, 1e-3, 1e-4)], 0.01)
    fan = np.vstack([tris, [[0, 1, len(X)]], [[0, 1, len(X) + 1]]]).astype(np.int32)  # edge (0, 1) in 3 triangles
    Xf = np.vstack([X, [[0.05, -0.05, 0.02]], [[0.05, -0.05, -0.02]]])
    with pytest.raises(pkg.NcpadjError, match="more than two"):
        pkg.Scene.shells(ctx, [(Xf, fan, np.full(len(fan), 1e5), np.full(len(fan), 0.3), 1000.0, 1e-3, 1e-4)], 0.01)
    scene = pkg.Scene.shells(ctx, [good], 0.01)
    with pytest.raises(pkg.NcpadjError, match="tet scenes"):
        scene.set_fibres(np.tile([1.0, 0.0, 0.0], (len(tris), 1)))
    with pytest.raises(pkg.NcpadjError, match="bend"):
        scene.set_bending(-1.0)
