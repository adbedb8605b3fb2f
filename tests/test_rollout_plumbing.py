"""The autograd plumbing of differentiable rollouts (CPU only): StepFn and rollout() with the
library's forward and adjoint calls replaced by a linear step and its exact transpose, so that
torch's own autograd through the same recurrence is the reference.  Covers the state chain,
f_ext, per-step and constant binding targets, binding compliances, and checkpointed segments."""
import types

import pytest
import torch

import paper_2603_16478_gb300.rollout as R

A, C1, C2, CB, CC, H = 0.9, 0.05, 0.01, 0.3, 0.7, 0.01
BV = torch.tensor([1, 4, 6], dtype=torch.int32)  # bound vertices
NV = 8


def _scatter(rows):
    out = torch.zeros(NV, 3, dtype=torch.float64)
    out.index_add_(0, BV.long(), rows)
    return out


def _step_torch(q_prev, v_prev, f_ext, target, compliance):
    """The fake step written with torch ops (the autograd reference)."""
    q = A * q_prev + C1 * v_prev + C2 * f_ext
    if target is not None:
        q = q + CB * _scatter(target) + CC * _scatter(compliance[:, None].expand(-1, 3))
    return q


def _fake_forward(scene, contacts, q_prev, v_prev, f_ext, gravity, *, bindings=None, **kw):
    f = f_ext if f_ext is not None else torch.zeros_like(q_prev)
    q = _step_torch(q_prev, v_prev, f, None if bindings is None else bindings.target,
                    None if bindings is None else bindings.compliance)
    return q, torch.zeros((0, 3), dtype=torch.float64), {"residual": 0.0}


def _fake_adjoint(scene, contacts, q, q_prev, lam, gq, gv, *, want=(), bindings=None, **kw):
    b = gq + gv / H
    g = {"dL_dq_prev": A * b - gv / H, "dL_dv_prev": C1 * b, "dL_dfext": C2 * b,
         "dL_dE": torch.zeros(5, dtype=torch.float64), "dL_dnu": torch.zeros(5, dtype=torch.float64),
         "dL_dmu": torch.zeros(1, dtype=torch.float64)}
    if bindings is not None:
        rows = b[bindings.vertex.long()]
        g["dL_dbinding_target"] = CB * rows
        g["dL_dcompliance"] = CC * rows.sum(dim=1)
    return g, {"iterations": 0}


class _FakeScene:
    """The scene's side of the material handling: its current per-tet material and the refactors asked for."""
    h, n_verts, n_tets = H, NV, 5

    def __init__(self):
        self.E = torch.full((5,), 1e5, dtype=torch.float64)
        self.nu = torch.full((5,), 0.4, dtype=torch.float64)
        self.refactors = []

    def material(self):
        return self.E.clone(), self.nu.clone()

    def refactor(self, E, nu):
        self.refactors.append((E, nu))
        self.E[:], self.nu[:] = E, nu


@pytest.fixture
def sim(monkeypatch):
    monkeypatch.setattr(R, "forward_step", _fake_forward)
    monkeypatch.setattr(R, "adjoint_step", _fake_adjoint)
    return R.Simulator(_FakeScene(), planes=[], binding_vertex=BV)


@pytest.mark.parametrize("ckpt", [0, 2])
def test_a_new_material_refactors_the_scene_once(sim, ckpt):
    """The factor is built for one material: E or nu different from the scene's refactor it before the
    first step, and only then (the steps and the backward recomputation share the material)."""
    n = 4
    q0 = torch.randn(NV, 3, dtype=torch.float64, requires_grad=True)
    v0 = torch.zeros(NV, 3, dtype=torch.float64)
    mu = torch.zeros(1, dtype=torch.float64)
    qT, _ = R.rollout(sim, q0, v0, torch.tensor(1e5, dtype=torch.float64), torch.tensor(0.4, dtype=torch.float64), mu,
                      n, checkpoint_every=ckpt)
    qT.sum().backward()
    assert sim.scene.refactors == []  # the scene's own material: nothing to rebuild
    qT, _ = R.rollout(sim, q0, v0, torch.tensor(2e5, dtype=torch.float64), torch.tensor(0.45, dtype=torch.float64),
                      mu, n, checkpoint_every=ckpt)
    qT.sum().backward()
    assert sim.scene.refactors == [(2e5, 0.45)]
    assert float(sim.scene.E[0]) == 2e5 and float(sim.scene.nu[3]) == 0.45


@pytest.mark.parametrize("ckpt", [0, 2])
@pytest.mark.parametrize("per_step", [True, False])
def test_rollout_gradients_match_autograd_of_the_same_recurrence(sim, ckpt, per_step):
    n = 5
    g = torch.Generator().manual_seed(0)
    mk = lambda *s: torch.randn(*s, generator=g, dtype=torch.float64)  # noqa: E731
    q0, v0, f = mk(NV, 3), mk(NV, 3), mk(NV, 3)
    tg = mk(n, len(BV), 3) if per_step else mk(len(BV), 3)
    comp = mk(len(BV)).abs() + 0.1
    w1, w2 = mk(NV, 3), mk(NV, 3)
    E, nu, mu = torch.tensor(1e5, dtype=torch.float64), torch.tensor(0.4, dtype=torch.float64), torch.zeros(1, dtype=torch.float64)

    def loss(run):
        ins = [x.clone().requires_grad_(True) for x in (q0, v0, f, tg, comp)]
        qT, vT = run(*ins)
        L = (qT * w1).sum() + (vT * w2).sum()
        return L, torch.autograd.grad(L, ins)

    def lib(q0_, v0_, f_, tg_, c_):
        return R.rollout(sim, q0_, v0_, E, nu, mu, n, checkpoint_every=ckpt, f_ext=f_, binding_targets=tg_,
                         binding_compliance=c_)

    def ref(q0_, v0_, f_, tg_, c_):
        q, v = q0_, v0_
        for t in range(n):
            qn = _step_torch(q, v, f_, tg_[t] if per_step else tg_, c_)
            q, v = qn, (qn - q) / H
        return q, v

    L1, g1 = loss(lib)
    L2, g2 = loss(ref)
    assert torch.allclose(L1, L2, rtol=1e-12)
    for name, a, b in zip(("q0", "v0", "f_ext", "targets", "compliance"), g1, g2):
        assert torch.allclose(a, b, rtol=1e-10, atol=1e-10), name


def test_rollout_without_bindings_is_unchanged(sim):
    n = 3
    q0 = torch.randn(NV, 3, dtype=torch.float64, requires_grad=True)
    v0 = torch.zeros(NV, 3, dtype=torch.float64)
    E, nu, mu = torch.tensor(1e5, dtype=torch.float64), torch.tensor(0.4, dtype=torch.float64), torch.zeros(1, dtype=torch.float64)
    qT, vT = R.rollout(sim, q0, v0, E, nu, mu, n)
    qT.sum().backward()
    # the plain chain: dq_T/dq0 for v0 = 0 follows q_{t+1} = A q_t + C1 (q_t - q_{t-1}) / H
    q, v = q0.detach().clone().requires_grad_(True), v0
    qq, vv = q, v
    for _ in range(n):
        qn = A * qq + C1 * vv
        qq, vv = qn, (qn - qq) / H
    (g_ref,) = torch.autograd.grad(qq.sum(), q)
    assert torch.allclose(q0.grad, g_ref, rtol=1e-12)


def test_per_step_targets_need_one_slice_per_step(sim):
    E, nu, mu = torch.tensor(1e5), torch.tensor(0.4), torch.zeros(1)
    with pytest.raises(ValueError):
        R.rollout(sim, torch.zeros(NV, 3, dtype=torch.float64), torch.zeros(NV, 3, dtype=torch.float64), E, nu, mu, 3,
                  binding_targets=torch.zeros(2, len(BV), 3, dtype=torch.float64),
                  binding_compliance=torch.ones(len(BV), dtype=torch.float64))


def test_simulator_contact_detection_matches_the_input_generator():
    """Simulator.contacts (torch, used by rollouts) selects the same vertices with the same frames,
    offsets and per-region friction as synth.detect_contacts for planes without region grids."""
    import numpy as np

    import synth
    pb = synth.beam_incline(nx=8, ny=3, nz=3)
    sc = pb.scene
    q = torch.as_tensor(pb.q0)
    planes = [R.PlaneCollider(p.normal.tolist(), p.offset, p.t1.tolist(), p.t2.tolist(), region=i)
              for i, p in enumerate(sc.planes)]
    ref_planes = [synth.Plane(p.normal, p.offset, mu) for p, mu in zip(sc.planes, (0.3, 0.7))]
    for rp, p in zip(ref_planes, sc.planes):
        rp.t1, rp.t2 = p.t1, p.t2
    sim = R.Simulator(types.SimpleNamespace(h=sc.h), planes, margin=2e-3, n_regions=len(planes))
    mu_region = torch.tensor([0.3, 0.7][:len(planes)], dtype=torch.float64)
    got = sim.contacts(q, mu_region)
    ref = synth.detect_contacts(pb.q0, ref_planes, 2e-3)
    assert got.n == ref.n > 0
    assert np.array_equal(got.vertex.numpy(), ref.vertex)
    assert np.allclose(got.frame.numpy(), ref.frame) and np.allclose(got.d_n.numpy(), ref.d_n)
    assert np.array_equal(got.region.numpy(), ref.region) and np.allclose(got.mu.numpy(), ref.mu)
