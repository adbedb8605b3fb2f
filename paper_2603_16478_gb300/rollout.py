"""Differentiable rollouts: one implicit step as a ``torch.autograd.Function`` whose backward is the
analytical adjoint (Sec. 4.1), chained over time with checkpointed forward recomputation.

The gradient flow across steps follows Sec. 4.1: the adjoint of step t turns the seeds dL/dq_t,
dL/dv_t into dL/dq_{t-1}, dL/dv_{t-1} (propagated to the previous step) and into contributions to
the parameter gradients (summed over steps).  Every call goes to the C-ABI library; this module
only detects vertex-plane contacts (a gap test) and moves tensors.

Bilateral bindings (Eq. binding) are given per rollout as vertices (or points inside tets) on the
simulator, with targets that may change every step and compliances; both get gradients, the
targets per step (control of attachments and cables) and the compliances summed over steps.

Memory: a step saves only its inputs (q_prev, v_prev) and recomputes its converged state with
the forward step when the backward pass reaches it.  ``rollout(..., checkpoint_every=k)`` also
wraps segments of k steps in ``torch.utils.checkpoint`` so that only segment boundaries stay
resident during the forward pass.
"""
from __future__ import annotations

from dataclasses import dataclass, field
from typing import List, Optional, Sequence

import torch
from torch.utils.checkpoint import checkpoint

from .binding import Bindings, Contacts, Scene, adjoint_step, forward_step


@dataclass
class PlaneCollider:
    """Rigid plane {x : normal . x = offset} with frame rows (normal, t1, t2) and a friction region."""
    normal: Sequence[float]
    offset: float
    t1: Sequence[float]
    t2: Sequence[float]
    region: int = 0


@dataclass
class Simulator:
    """A scene plus the settings of its contact detection and solver."""
    scene: Scene
    planes: List[PlaneCollider]
    candidates: Optional[torch.Tensor] = None  # int64 vertex ids that may touch a plane (None: all)
    margin: float = 2e-3
    eps: float = 1e-4
    gravity: Sequence[float] = (0.0, 0.0, -9.81)
    n_regions: int = 1
    precision: str = "fp64"
    cap_precision: str = "fp64"
    rtol: float = 1e-8
    newton_tol: float = 1e-10
    max_newton: int = 100
    _frames: dict = field(default_factory=dict)
    _material: Optional[tuple] = None  # (E, nu) the scene's factor is built for, when uniform
    # bilateral bindings: vertices [n_b] (int32), or points inside tets (tet ids [n_b] and
    # barycentric weights [n_b, 4]); their targets and compliances are rollout inputs
    binding_vertex: Optional[torch.Tensor] = None
    binding_tet: Optional[torch.Tensor] = None
    binding_bary: Optional[torch.Tensor] = None

    def bindings(self, target: Optional[torch.Tensor], compliance: Optional[torch.Tensor]) -> Optional[Bindings]:
        if target is None:
            return None
        if compliance is None:
            raise ValueError("binding targets need compliances")
        return Bindings(self.binding_vertex, target.detach().contiguous(), compliance.detach().contiguous(),
                        tet=self.binding_tet, bary=self.binding_bary)

    def contacts(self, q_prev: torch.Tensor, mu_region: torch.Tensor) -> Optional[Contacts]:
        """Vertices whose gap at q_prev is below the margin, one contact per (vertex, plane)."""
        dev = q_prev.device
        verts = torch.arange(q_prev.shape[0], device=dev) if self.candidates is None else self.candidates.to(dev)
        vs, frames, dn, regs = [], [], [], []
        for pl in self.planes:
            n = torch.tensor(pl.normal, dtype=torch.float64, device=dev)
            gap = q_prev[verts] @ n - pl.offset
            sel = verts[gap < self.margin]
            if sel.numel() == 0:
                continue
            fr = torch.stack([n, torch.tensor(pl.t1, dtype=torch.float64, device=dev),
                              torch.tensor(pl.t2, dtype=torch.float64, device=dev)])
            vs.append(sel)
            frames.append(fr.expand(sel.numel(), 3, 3))
            dn.append(torch.full((sel.numel(),), float(pl.offset), dtype=torch.float64, device=dev))
            regs.append(torch.full((sel.numel(),), pl.region, dtype=torch.int32, device=dev))
        if not vs:
            return None
        region = torch.cat(regs)
        return Contacts(torch.cat(vs).to(torch.int32).contiguous(), torch.cat(frames).contiguous(),
                        torch.cat(dn).contiguous(), mu_region.detach()[region.long()].contiguous(), None,
                        region.contiguous(), self.n_regions)

    def use_material(self, E, nu) -> None:
        """Make the scene's elastic factor the one of the uniform material (E, nu): the scene is
        refactored (ncpadj_scene_refactor) when its current material differs."""
        want = (float(E), float(nu))
        if self._material is None:
            e, n = self.scene.material()
            if bool((e == e[0]).all()) and bool((n == n[0]).all()):
                self._material = (float(e[0]), float(n[0]))
        if self._material != want:
            self.scene.refactor(want[0], want[1])
            self._material = want

    def step(self, q_prev, v_prev, contacts, f_ext=None, act=None, bindings=None):
        return forward_step(self.scene, contacts, q_prev.contiguous(), v_prev.contiguous(), f_ext, self.gravity,
                            eps=self.eps, newton_tol=self.newton_tol, max_newton=self.max_newton,
                            act=None if act is None else act.detach().contiguous(), bindings=bindings)


class StepFn(torch.autograd.Function):
    """(q_prev, v_prev, E, nu, mu_region, f_ext, act, b_target, b_compliance) -> (q, v) for one
    implicit step.

    E and nu are scalar tensors: the uniform material of the step.  The scene's elastic factor is
    built for one material, so the forward pass (and the backward pass, which recomputes the step)
    first refactors the scene when its material differs; the backward pass returns dL/dE and
    dL/dnu summed over tets.  mu_region [n_regions] sets every contact's
    friction coefficient through its region.  act (FP32 [n_tets] or None) are the per-tet
    activations of the scene's fibres (constant active stress a_i d_i d_i^T).  b_target [n_b, 3]
    and b_compliance [n_b] (or None) are the step's bilateral bindings on the simulator's
    binding vertices or points.
    """

    @staticmethod
    def forward(ctx, q_prev, v_prev, E, nu, mu_region, f_ext, act, b_target, b_compliance, sim: Simulator):
        sim.use_material(E, nu)
        ctx.material = (float(E), float(nu))
        contacts = sim.contacts(q_prev, mu_region)
        q, lam, _ = sim.step(q_prev, v_prev, contacts, f_ext, act, sim.bindings(b_target, b_compliance))
        v = (q - q_prev) / sim.scene.h
        ctx.sim = sim
        ctx.has_fext = f_ext is not None
        ctx.has_act = act is not None
        ctx.has_bind = b_target is not None
        # save the inputs only: the converged state is recomputed in backward
        empty = torch.empty(0)
        ctx.save_for_backward(q_prev, v_prev, mu_region, f_ext if f_ext is not None else empty,
                              act if act is not None else empty, b_target if b_target is not None else empty,
                              b_compliance if b_target is not None else empty)
        return q, v

    @staticmethod
    def backward(ctx, gq, gv):
        sim: Simulator = ctx.sim
        q_prev, v_prev, mu_region, f_ext, act, b_target, b_compliance = ctx.saved_tensors
        f_ext = f_ext if ctx.has_fext else None
        act = act if ctx.has_act else None
        bd = sim.bindings(b_target, b_compliance) if ctx.has_bind else None
        sim.use_material(*ctx.material)
        contacts = sim.contacts(q_prev, mu_region)
        q, lam, _ = sim.step(q_prev, v_prev, contacts, f_ext, act, bd)
        gq = torch.zeros_like(q) if gq is None else gq.contiguous()
        gv = torch.zeros_like(q) if gv is None else gv.contiguous()
        want = ("dL_dq_prev", "dL_dv_prev", "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu") + (("dL_dact",) if act is not None
                                                                                      else ())
        g, _ = adjoint_step(sim.scene, contacts, q, q_prev, lam.contiguous(), gq, gv, eps=sim.eps, rtol=sim.rtol,
                            precision=sim.precision, cap_precision=sim.cap_precision, want=want, bindings=bd)
        d_mu = g["dL_dmu"] if contacts is not None else torch.zeros_like(mu_region)
        d_f = g["dL_dfext"] if ctx.has_fext else None
        d_a = g["dL_dact"] if act is not None else None
        d_bt = g["dL_dbinding_target"] if bd is not None else None
        d_bc = g["dL_dcompliance"] if bd is not None else None
        return (g["dL_dq_prev"], g["dL_dv_prev"], g["dL_dE"].sum(), g["dL_dnu"].sum(), d_mu, d_f, d_a, d_bt, d_bc,
                None)


def rollout(sim: Simulator, q0, v0, E, nu, mu_region, n_steps: int, checkpoint_every: int = 0, f_ext=None,
            act=None, binding_targets=None, binding_compliance=None):
    """Run n_steps differentiable steps; returns (q_T, v_T).  With checkpoint_every = k > 0 the steps
    are grouped in segments of k under torch.utils.checkpoint (forward recomputed in backward).
    ``act``: per-tet activations (FP32 [n_tets]) applied at every step (the scene needs fibres).
    ``binding_targets``: [n_b, 3] for every step, or [n_steps, n_b, 3] one per step, with
    ``binding_compliance`` [n_b] (the simulator names the bound vertices or points)."""
    q, v = q0, v0
    if binding_targets is not None and binding_targets.dim() == 3 and binding_targets.shape[0] != n_steps:
        raise ValueError("per-step binding targets need one [n_b, 3] slice per step")

    def target_at(bt, t):
        if bt is None:
            return None
        return bt if bt.dim() == 2 else bt[t]

    def segment(q_, v_, E_, nu_, mu_, k, act_, t0, bt, bc):
        for i in range(k):
            q_, v_ = StepFn.apply(q_, v_, E_, nu_, mu_, f_ext, act_, target_at(bt, t0 + i), bc, sim)
        return q_, v_

    t = 0
    while t < n_steps:
        k = min(checkpoint_every, n_steps - t) if checkpoint_every > 0 else 1
        if checkpoint_every > 0:
            q, v = checkpoint(segment, q, v, E, nu, mu_region, k, act, t, binding_targets, binding_compliance,
                              use_reentrant=False)
        else:
            q, v = segment(q, v, E, nu, mu_region, 1, act, t, binding_targets, binding_compliance)
        t += k
    return q, v
