"""Multi-step gradients through the torch.autograd.Function rollout match the oracle's chain of
one-step adjoints (Sec. 4.1: state gradients propagate to the previous step, parameter gradients
accumulate), with and without checkpointed segments."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from tests._cases import make_step, rel  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


def _sim(pkg, pb, **kw):
    from paper_2603_16478_gb300.rollout import PlaneCollider, Simulator
    sc = pb.scene
    ctx = pkg.Context(0)
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    planes = [PlaneCollider(tuple(p.normal), p.offset, tuple(p.t1), tuple(p.t2), i) for i, p in enumerate(sc.planes)]
    sim = Simulator(scene, planes, torch.as_tensor(sc.contact_candidates, device="cuda"), sc.margin, sc.eps,
                    tuple(sc.gravity), n_regions=len(sc.planes), **kw)
    sim._ctx = ctx
    return sim


def _loss(q, tgt):
    return ((q.mean(0) - tgt) ** 2).sum()


def _oracle_chain(pb, n_steps, tgt):
    sc = pb.scene
    q_prev, v_prev = pb.q0.copy(), pb.v0.copy()
    steps = []
    for _ in range(n_steps):
        ct = sc.contacts(q_prev)
        st = make_step(sc, ct)
        s = st.forward(q_prev, v_prev)
        steps.append((st, s, q_prev))
        v_prev = (s.q - q_prev) / sc.h
        q_prev = s.q
    gq = 2 * (q_prev.mean(0) - tgt)[None, :].repeat(sc.n_verts, 0) / sc.n_verts
    gv = np.zeros_like(gq)
    dE = dnu = 0.0
    dmu = np.zeros(len(sc.planes))
    for st, s, qp in reversed(steps):
        g = st.adjoint(s, qp, gq, gv)
        dE += g["dL_dE"].sum()
        dnu += g["dL_dnu"].sum()
        dmu += g["dL_dmu_region"]
        gq, gv = g["dL_dq_prev"], g["dL_dv_prev"]
    return dict(E=dE, nu=dnu, mu=dmu, q0=gq, v0=gv)


@pytest.mark.parametrize("ckpt", [0, 2])
def test_rollout_gradients_match_oracle_chain(pkg, ckpt):
    from paper_2603_16478_gb300.rollout import rollout
    pb = synth.beam_incline(nx=6, ny=3, nz=2)
    sc = pb.scene
    n_steps = 4
    tgt = pb.q0.mean(0) + 1e-3 * np.asarray(sc.planes[0].t1)
    ref = _oracle_chain(pb, n_steps, tgt)
    sim = _sim(pkg, pb)
    dev = "cuda"
    q0 = torch.as_tensor(pb.q0, device=dev).requires_grad_(True)
    v0 = torch.as_tensor(pb.v0, device=dev).requires_grad_(True)
    E = torch.tensor(float(sc.E[0]), dtype=torch.float64, device=dev, requires_grad=True)
    nu = torch.tensor(float(sc.nu[0]), dtype=torch.float64, device=dev, requires_grad=True)
    mu = torch.tensor([p.mu for p in sc.planes], dtype=torch.float64, device=dev, requires_grad=True)
    qT, vT = rollout(sim, q0, v0, E, nu, mu, n_steps, checkpoint_every=ckpt)
    L = _loss(qT, torch.as_tensor(tgt, device=dev))
    L.backward()
    assert rel(E.grad.item(), ref["E"]) < 1e-5
    assert rel(nu.grad.item(), ref["nu"]) < 1e-5
    assert rel(mu.grad.cpu().numpy(), ref["mu"]) < 1e-5
    assert rel(q0.grad.cpu().numpy(), ref["q0"]) < 1e-5
    assert rel(v0.grad.cpu().numpy(), ref["v0"]) < 1e-5


def test_beam_rollout_30_steps_mixed_vs_fp64(pkg):
    """Full-size beam (20k tets), 30 steps at h = 1/100, gradients of the final centre-of-mass error
    w.r.t. E, nu and mu through the autograd rollout (checkpoint every step): mixed vs FP64."""
    from paper_2603_16478_gb300.rollout import rollout
    pb = synth.beam_incline()
    sc = pb.scene
    tgt = torch.as_tensor(pb.q0.mean(0) + 5e-3 * np.asarray(sc.planes[0].t1), device="cuda")
    grads = {}
    for prec in ("fp64", "mixed"):
        sim = _sim(pkg, pb, precision=prec, cap_precision=prec)
        E = torch.tensor(float(sc.E[0]), dtype=torch.float64, device="cuda", requires_grad=True)
        nu = torch.tensor(float(sc.nu[0]), dtype=torch.float64, device="cuda", requires_grad=True)
        mu = torch.tensor([p.mu for p in sc.planes], dtype=torch.float64, device="cuda", requires_grad=True)
        qT, _ = rollout(sim, torch.as_tensor(pb.q0, device="cuda"), torch.as_tensor(pb.v0, device="cuda"), E, nu, mu,
                        30, checkpoint_every=1)
        _loss(qT, tgt).backward()
        grads[prec] = np.array([E.grad.item(), nu.grad.item(), *mu.grad.cpu().numpy()])
    assert np.all(np.isfinite(grads["fp64"]))
    assert rel(grads["mixed"], grads["fp64"]) < 1e-3, grads


def test_quadruped_rollout_activation_gradient_matches_oracle_chain(pkg):
    """Down-scaled soft quadruped (voxel torso, legs and foot pads; 192 pad contacts, mu = 0.8),
    2 steps at h = 1/200 with seeded per-tet activations (N(0, 200^2) Pa): dL/da of
    L = -mean x(q_T) through the autograd rollout against the oracle's chain of one-step adjoints."""
    from oracle.actuation import actuation_force, actuation_gradient
    from paper_2603_16478_gb300.rollout import rollout
    pb = synth.quadruped(torso=(16, 10, 2), leg_r=2.0, leg_h=3, leg_c=(5, 3), pad=(7, 5, 1), cell=0.02,
                         act_scale=2e2)
    sc = pb.scene
    n_steps = 2
    act, fibre = pb.act.astype(np.float32), pb.fibre
    # oracle chain
    q_prev, v_prev = pb.q0.copy(), pb.v0.copy()
    steps = []
    for _ in range(n_steps):
        ct = sc.contacts(q_prev)
        st = make_step(sc, ct)
        s = st.forward(q_prev, v_prev, f_ctrl=actuation_force(st.mesh, act.astype(float), fibre))
        assert s.residual < 1e-8
        steps.append((st, s, q_prev))
        v_prev = (s.q - q_prev) / sc.h
        q_prev = s.q
    gq = np.zeros_like(q_prev)
    gq[:, 0] = -1.0 / sc.n_verts
    gv = np.zeros_like(gq)
    da = np.zeros(sc.n_tets)
    for st, s, qp in reversed(steps):
        g = st.adjoint(s, qp, gq, gv)
        da += actuation_gradient(st.mesh, g["z"], fibre, sc.h)
        gq, gv = g["dL_dq_prev"], g["dL_dv_prev"]
    sim = _sim(pkg, pb)
    sim.scene.set_fibres(fibre)
    a = torch.as_tensor(act, device="cuda").requires_grad_(True)
    E = torch.tensor(float(sc.E[0]), dtype=torch.float64, device="cuda")
    nu = torch.tensor(float(sc.nu[0]), dtype=torch.float64, device="cuda")
    mu = torch.tensor([p.mu for p in sc.planes], dtype=torch.float64, device="cuda")
    qT, _ = rollout(sim, torch.as_tensor(pb.q0, device="cuda"), torch.as_tensor(pb.v0, device="cuda"), E, nu, mu,
                    n_steps, checkpoint_every=1, act=a)
    (-qT[:, 0].mean()).backward()
    assert rel(a.grad.double().cpu().numpy(), da) < 1e-4
