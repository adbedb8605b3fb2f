"""Per-tet muscle actuation as a constant active stress (test infrastructure: oracle).

The paper drives its soft robots with muscles it describes only in words (Sec. 5, the seal
rollout).  The reading used here: tet i carries a scalar activation a_i and a fixed unit fibre
direction d_i in the rest frame; the activation adds the constant first Piola-Kirchhoff stress
    P_act,i = a_i d_i d_i^T,
whose nodal force is the negative gradient of the work V_i P_act,i : F_i(q), i.e.
    f_act = - sum_i V_i G_i^T vec(P_act,i)                              (G_i of Sec. 3.1).
The force does not depend on q, so the adjoint matrix is unchanged and the activation enters
the step only through f_ext (qtilde = qbar + h vbar + h^2 M^{-1} f_ext).  With dL/df_ext = h^2 z
(Eq. compute_gradient),
    dL/da_i = h^2 z^T df_act/da_i = - h^2 V_i (G_i z) . vec(d_i d_i^T) = - h^2 V_i d_i^T Z_i d_i,
where Z_i = unvec(G_i z) is the "deformation gradient" of the adjoint field z on tet i.
"""
from __future__ import annotations

import numpy as np

from .model import Mesh, vec


def stress_force(mesh: Mesh, P):
    """Nodal forces [n_v, 3] of constant per-tet first Piola stresses P [n_t, 3, 3]:
    f = - sum_i V_i G_i^T vec(P_i)."""
    per_tet = -mesh.vol[:, None] * np.einsum("tij,ti->tj", mesh.G, vec(np.asarray(P, float)))
    return mesh.scatter_vectors(per_tet).reshape(-1, 3)


def active_stress(act, fibre):
    """P_act,i = a_i d_i d_i^T  [n_t, 3, 3]."""
    d = np.asarray(fibre, float)
    return np.asarray(act, float)[:, None, None] * np.einsum("ti,tj->tij", d, d)


def actuation_force(mesh: Mesh, act, fibre):
    """f_act [n_v, 3] for activations a [n_t] and unit fibres d [n_t, 3]."""
    return stress_force(mesh, active_stress(act, fibre))


def actuation_gradient(mesh: Mesh, z, fibre, h):
    """dL/da [n_t] from the adjoint solution z [n_v, 3]."""
    d = np.asarray(fibre, float)
    Gz = mesh.Gx(np.asarray(z, float).reshape(-1))               # vec(Z_i) [n_t, 9]
    ddT = vec(np.einsum("ti,tj->tij", d, d))
    return -h * h * mesh.vol * np.sum(Gz * ddT, axis=1)
