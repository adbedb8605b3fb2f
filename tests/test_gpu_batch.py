"""The batched adjoint (one call over the disjoint union of several scenes) gives each scene the
same gradients as its own single-scene adjoint, and the oracle's."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from tests._cases import rel, step_case  # noqa: E402
from tests.test_gpu_parity import KEYS, T  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


def _cases():
    # three scenes with contacts of different kinds + one without contacts
    return [step_case("cube_drop", 2), step_case("two_tet", 1), step_case("cube_drop", 5), step_case("cube_drop", 0)]


@pytest.mark.parametrize("side_stream", [False, True])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_batch_equals_single_scene_adjoints(pkg, precision, side_stream):
    """On a side stream the GMRES steps are replays of a captured graph (several capacitance
    blocks in one step); on the default stream the same kernels are launched one by one."""
    ctx = pkg.Context(0)
    cases = _cases()
    rng = np.random.default_rng(0)
    meshes, seeds, refs = [], [], []
    for pb, st, s, q_prev, v_prev in cases:
        sc = pb.scene
        meshes.append((sc.X, sc.tets, sc.E, sc.nu, sc.density))
        dq = rng.normal(size=s.q.shape) * 10.0 ** rng.uniform(-3, 3)  # scenes with very different seed scales
        dv = rng.normal(size=s.q.shape) * 1e-3
        seeds.append((dq, dv))
        refs.append(st.adjoint(s, q_prev, dq, dv))
    batch = pkg.Scene.batch(ctx, meshes, cases[0][0].scene.h)
    off = batch.vertex_offsets
    vert, frame, dn, mu, region, lam, q, qp, dqs, dvs = [], [], [], [], [], [], [], [], [], []
    nreg = 0
    for i, ((pb, st, s, q_prev, v_prev), (dq, dv)) in enumerate(zip(cases, seeds)):
        ct = st.ct
        vert.append(ct.vertex + off[i])
        frame.append(ct.frame)
        dn.append(ct.d_n)
        mu.append(ct.mu)
        region.append(ct.region + nreg)
        nreg += ct.n_regions
        lam.append(s.lam_frame(st, q_prev) if ct.n else np.zeros((0, 3)))
        q.append(s.q)
        qp.append(q_prev)
        dqs.append(dq)
        dvs.append(dv)
    contacts = pkg.Contacts(T(np.concatenate(vert), torch.int32), T(np.concatenate(frame)), T(np.concatenate(dn)),
                            T(np.concatenate(mu)), None, T(np.concatenate(region), torch.int32), nreg)
    stream = torch.cuda.Stream() if side_stream else None
    torch.cuda.synchronize()
    g, stats = pkg.adjoint_step(batch, contacts, T(np.concatenate(q)), T(np.concatenate(qp)), T(np.concatenate(lam)),
                                T(np.concatenate(dqs)), T(np.concatenate(dvs)), eps=cases[0][0].scene.eps,
                                rtol=1e-12 if precision == "fp64" else 1e-8, precision=precision,
                                cap_precision=precision, stream=None if stream is None else stream.cuda_stream)
    torch.cuda.synchronize()
    tol = 1e-8 if precision == "fp64" else 1e-3
    toff = batch.tet_offsets
    c0 = 0
    r0 = 0
    for i, ((pb, st, s, q_prev, v_prev), ref) in enumerate(zip(cases, refs)):
        sl_v = slice(off[i], off[i + 1])
        for k in ("dL_dq_prev", "dL_dv_prev", "dL_dfext", "z"):
            assert rel(g[k][sl_v].cpu().numpy(), ref[k]) <= tol, (i, k)
        for k in ("dL_dE", "dL_dnu"):
            assert rel(g[k][toff[i]:toff[i + 1]].cpu().numpy(), ref[k]) <= tol, (i, k)
        nci = st.ct.n
        if nci:
            assert rel(g["dL_dmu_contact"][c0:c0 + nci].cpu().numpy(), ref["dL_dmu_contact"]) <= tol, (i, "mu_c")
            assert rel(g["dL_dmu"][r0:r0 + st.ct.n_regions].cpu().numpy(), ref["dL_dmu_region"]) <= tol, (i, "mu")
        c0 += nci
        r0 += st.ct.n_regions


def test_batch_rejects_ungrouped_contacts(pkg):
    ctx = pkg.Context(0)
    cases = _cases()[:2]
    batch = pkg.Scene.batch(ctx, [(c[0].scene.X, c[0].scene.tets, c[0].scene.E, c[0].scene.nu, c[0].scene.density)
                                  for c in cases], cases[0][0].scene.h)
    off = batch.vertex_offsets
    (pa, sa, xa, qa, _), (pb_, sb, xb, qb, _) = cases
    vert = np.concatenate([sb.ct.vertex + off[1], sa.ct.vertex + off[0]])  # scene 1 before scene 0
    frame = np.concatenate([sb.ct.frame, sa.ct.frame])
    n = len(vert)
    contacts = pkg.Contacts(T(vert, torch.int32), T(frame), T(np.zeros(n)), T(np.full(n, 0.5)), None,
                            T(np.zeros(n), torch.int32), 1)
    q = T(np.concatenate([xa.q, xb.q]))
    lam = T(np.concatenate([xb.lam_frame(sb, qb), xa.lam_frame(sa, qa)]))
    with pytest.raises(pkg.NcpadjError, match="grouped by scene"):
        pkg.adjoint_step(batch, contacts, q, T(np.concatenate([qa, qb])), lam, torch.ones_like(q), None)


def test_batched_forward_reaches_every_scenes_own_state(pkg):
    """One forward call over a batch (per-scene line searches) converges every scene to the state its
    own single-scene forward reaches, including scenes that need heavily damped steps."""
    ctx = pkg.Context(0)
    from tests._cases import rollout
    starts = [rollout("cube_drop", 2), rollout("two_tet", 1), rollout("cube_drop", 5), rollout("cube_drop", 0),
              rollout("cube_drop", 4)]
    meshes, singles = [], []
    for pb, q_prev, v_prev in starts:
        sc = pb.scene
        meshes.append((sc.X, sc.tets, sc.E, sc.nu, sc.density))
        scene1 = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
        ct = sc.contacts(q_prev)
        c1 = None if ct.n == 0 else pkg.Contacts(T(ct.vertex, torch.int32), T(ct.frame), T(ct.d_n), T(ct.mu),
                                                  None, T(ct.region, torch.int32), ct.n_regions)
        q1, _, st1 = pkg.forward_step(scene1, c1, T(q_prev), T(v_prev), None, tuple(sc.gravity), eps=sc.eps,
                                      newton_tol=1e-11)
        singles.append((q1.cpu().numpy(), ct))
    batch = pkg.Scene.batch(ctx, meshes, starts[0][0].scene.h)
    off = batch.vertex_offsets
    vert, frame, dn, mu, region = [], [], [], [], []
    for i, (q1, ct) in enumerate(singles):
        vert.append(ct.vertex + off[i])
        frame.append(ct.frame)
        dn.append(ct.d_n)
        mu.append(ct.mu)
        region.append(np.full(ct.n, i, np.int32))
    contacts = pkg.Contacts(T(np.concatenate(vert), torch.int32), T(np.concatenate(frame)), T(np.concatenate(dn)),
                            T(np.concatenate(mu)), None, T(np.concatenate(region), torch.int32), len(starts))
    q0 = T(np.concatenate([s[1] for s in starts]))
    v0 = T(np.concatenate([s[2] for s in starts]))
    qb, lamb, stb = pkg.forward_step(batch, contacts, q0, v0, None, tuple(starts[0][0].scene.gravity),
                                     eps=starts[0][0].scene.eps, newton_tol=1e-11, max_newton=120)
    qb = qb.cpu().numpy()
    for i, ((q1, _), (pb, q_prev, _)) in enumerate(zip(singles, starts)):
        seg = qb[off[i]:off[i + 1]]
        assert rel(seg - q_prev, q1 - q_prev) < 1e-7, (i, rel(seg - q_prev, q1 - q_prev))


def _batch_inputs(cases, rng, zero_seed=None):
    """Per-scene inputs of the batch cases in each scene's own numbering (numpy), and the oracle
    references; scene zero_seed (if given) gets a zero loss seed."""
    per, refs = [], []
    for i, (pb, st, s, q_prev, v_prev) in enumerate(cases):
        dq = rng.normal(size=s.q.shape) * 10.0 ** rng.uniform(-3, 3)
        dv = rng.normal(size=s.q.shape) * 1e-3
        if i == zero_seed:
            dq, dv = np.zeros_like(dq), np.zeros_like(dv)
        lam = s.lam_frame(st, q_prev) if st.ct.n else np.zeros((0, 3))
        per.append((st.ct, s.q, q_prev, lam, dq, dv))
        refs.append(st.adjoint(s, q_prev, dq, dv))
    return per, refs


def _uneven_cases():
    # scenes of different sizes and contact regimes, so their own GMRES needs different counts
    return [step_case("cube_drop", 2), step_case("two_tet", 1), step_case("cube_drop", 5), step_case("cube_drop", 0),
            step_case("cube_drop", 3)]


@pytest.mark.parametrize("memory", ["device", "host"])
@pytest.mark.parametrize("precision", ["fp64", "mixed"])
def test_adjoint_batch_matches_oracle_scene_by_scene(pkg, precision, memory):
    """ncpadj_adjoint_batch: per-scene arrays in and out; every scene equals the oracle and stops at
    its own iteration count (about its single-scene count), not at the slowest scene's."""
    from tests.test_gpu_parity import gpu_contacts
    ctx = pkg.Context(0)
    cases = _uneven_cases()
    rng = np.random.default_rng(1)
    per, refs = _batch_inputs(cases, rng, zero_seed=3)
    batch = pkg.Scene.batch(ctx, [(c[0].scene.X, c[0].scene.tets, c[0].scene.E, c[0].scene.nu, c[0].scene.density)
                                  for c in cases], cases[0][0].scene.h)
    dev = "cuda" if memory == "device" else "cpu"
    rtol = 1e-12 if precision == "fp64" else 1e-8
    cts = [gpu_contacts(pkg, ct, dev) for ct, *_ in per]
    outs, stats = pkg.adjoint_batch(batch, cts, [T(p[1], dev=dev) for p in per], [T(p[2], dev=dev) for p in per],
                                    [T(p[3], dev=dev) for p in per], [T(p[4], dev=dev) for p in per],
                                    [T(p[5], dev=dev) for p in per], eps=cases[0][0].scene.eps, rtol=rtol,
                                    precision=precision, cap_precision=precision, memory=memory)
    torch.cuda.synchronize()
    tol = 1e-8 if precision == "fp64" else 1e-3
    for i, ((pb, st, s, q_prev, v_prev), ref, o, stt) in enumerate(zip(cases, refs, outs, stats)):
        for k in ("dL_dq_prev", "dL_dv_prev", "dL_dfext", "z", "dL_dE", "dL_dnu"):
            if i == 3:
                assert float(o[k].abs().max()) == 0.0, (i, k)
            else:
                assert rel(o[k].cpu().numpy(), ref[k]) <= tol, (i, k, rel(o[k].cpu().numpy(), ref[k]))
        if st.ct.n and i != 3:
            assert rel(o["dL_dmu_contact"].cpu().numpy(), ref["dL_dmu_contact"]) <= tol, (i, "mu_c")
            assert rel(o["dL_dmu"].cpu().numpy(), ref["dL_dmu_region"]) <= tol, (i, "mu")
        assert stt["rel_residual"] <= rtol * 1.0000001, (i, stt)
        assert stt["n_contacts"] == st.ct.n
    its = [s_["iterations"] for s_ in stats]
    assert its[3] == 0, its  # a zero seed is solved by z = 0 without an iteration
    assert len(set(its)) > 2, its  # each scene stops at its own count
    # each scene's count is its own GMRES's: the same scene alone (GMRES, same options) takes as many
    for i, (pb, st, s, q_prev, v_prev) in enumerate(cases):
        if i == 3:
            continue
        sc = pb.scene
        single = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
        ct, q, qp, lam, dq, dv = per[i]
        _, s1 = pkg.adjoint_step(single, gpu_contacts(pkg, ct), T(q), T(qp), T(lam), T(dq), T(dv), eps=sc.eps,
                                 rtol=rtol, precision=precision, cap_precision=precision, solver="gmres")
        assert abs(s1["iterations"] - its[i]) <= 2, (i, s1["iterations"], its[i])


def test_adjoint_batch_rejects_a_vertex_of_another_scene(pkg):
    from tests.test_gpu_parity import gpu_contacts
    ctx = pkg.Context(0)
    cases = _uneven_cases()[:2]
    per, _ = _batch_inputs(cases, np.random.default_rng(2))
    batch = pkg.Scene.batch(ctx, [(c[0].scene.X, c[0].scene.tets, c[0].scene.E, c[0].scene.nu, c[0].scene.density)
                                  for c in cases], cases[0][0].scene.h)
    cts = [gpu_contacts(pkg, ct) for ct, *_ in per]
    nv0 = cases[0][0].scene.X.shape[0]
    cts[0].vertex[0] = nv0  # one past scene 0's vertices: a vertex of scene 1 in the union
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        pkg.adjoint_batch(batch, cts, [T(p[1]) for p in per], [T(p[2]) for p in per], [T(p[3]) for p in per],
                          [T(p[4]) for p in per], None)


def test_adjoint_batch_reports_not_converged_per_scene(pkg):
    from tests.test_gpu_parity import gpu_contacts
    ctx = pkg.Context(0)
    cases = _uneven_cases()[:3]
    per, _ = _batch_inputs(cases, np.random.default_rng(3))
    batch = pkg.Scene.batch(ctx, [(c[0].scene.X, c[0].scene.tets, c[0].scene.E, c[0].scene.nu, c[0].scene.density)
                                  for c in cases], cases[0][0].scene.h)
    cts = [gpu_contacts(pkg, ct) for ct, *_ in per]
    with pytest.raises(pkg.NcpadjError, match="NOT_CONVERGED") as ei:
        pkg.adjoint_batch(batch, cts, [T(p[1]) for p in per], [T(p[2]) for p in per], [T(p[3]) for p in per],
                          [T(p[4]) for p in per], [T(p[5]) for p in per], rtol=1e-12, max_iters=3)
    st = ei.value.stats
    assert all(s_["iterations"] <= 3 for s_ in st), st
    assert max(s_["rel_residual"] for s_ in st) > 1e-12
    for o in ei.value.grads:  # the last iterate is still delivered
        assert torch.isfinite(o["z"]).all()
