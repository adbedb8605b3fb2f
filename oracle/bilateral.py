"""The equality-constrained (bilateral, frictionless) step and its adjoint, by dense LU
(test infrastructure: oracle).

As the smoothing eps of the Fischer-Burmeister contact goes to 0, a resting frictionless contact
(lambda_n > 0) enforces delta_n = n_c . q_v - d_n = 0 exactly.  The limit of the smoothed step is
therefore the solution of the KKT system
    R_q(q) / h^2 - N^T lam = 0,      N q - d = 0,
where R_q is the momentum residual without contacts (Eq. dynamics) and row c of N holds n_c at
vertex v_c.  Its adjoint, for a seed b = dL/dq + dL/dv / h, solves the transposed KKT matrix:
    [A_el/h^2  -N^T]^T [w_q]   [b]
    [N          0  ]   [w_l] = [0],      z* = w_q / h^2,
so that A_el^T z* + N^T w_l = b and N z* = 0 -- the limit of script_A^T z = b, script_A =
A_el + h^2 J^T K J, whose contact stiffness grows without bound as eps -> 0.  Every gradient
of Eq. (compute_gradient) is linear in z, so z* fixes the limit of all of them.
"""
from __future__ import annotations

import dataclasses

import numpy as np

from .step import State, Step


def _free(step: Step) -> Step:
    """The same scene with no contacts and no bindings."""
    ct = step.ct
    empty = dataclasses.replace(ct, vertex=ct.vertex[:0], frame=ct.frame[:0], d_n=ct.d_n[:0], d_f=ct.d_f[:0],
                                mu=ct.mu[:0], region=ct.region[:0])
    X = step.mesh.X
    return Step(X, step.mesh.tets, step.E, step.nu, step.density, step.h, step.gravity, empty, step.eps,
                step.model)


def vertex_rows(n_verts, vertex):
    """Rows selecting the coordinates of the given vertices [3 len(vertex), 3 n_verts] (the
    constraint rows of hard attachments q_v = d)."""
    Nm = np.zeros((3 * len(vertex), 3 * n_verts))
    for b, v in enumerate(vertex):
        Nm[3 * b:3 * b + 3, 3 * v:3 * v + 3] = np.eye(3)
    return Nm


def _normals(step: Step) -> np.ndarray:
    Nm = np.zeros((step.nc, step.N))
    for c in range(step.nc):
        v = step.ct.vertex[c]
        Nm[c, 3 * v:3 * v + 3] = step.ct.frame[c][0]
    return Nm


def constrained_step(step: Step, q_prev, v_prev, q_init, tol=1e-13, max_iter=50, Nm=None, d=None):
    """(q*, lam*) of the step with every contact of ``step`` held at delta_n = 0 (or, given Nm and
    d, with N q = d), by Newton's method on the KKT system with a dense LU, starting from q_init."""
    free = _free(step)
    if Nm is None:
        Nm, d = _normals(step), step.ct.d_n
    d = np.asarray(d, float).reshape(-1)
    N = step.N
    qt = free.qtilde(q_prev, v_prev, np.zeros_like(q_prev))
    q = np.asarray(q_init, float).copy()
    lam = np.zeros(Nm.shape[0])
    empty = np.zeros(0)
    for _ in range(max_iter):
        Rq = free.residual(q, empty, empty, q_prev, qt)[:N]
        F = np.concatenate([Rq - Nm.T @ lam, Nm @ q.reshape(-1) - d])
        if np.max(np.abs(F)) <= tol * (1.0 + np.max(np.abs(Rq - Rq.mean()))):
            break
        A_el, _ = free.adjoint_matrix(State(q, empty, empty), q_prev)
        m = Nm.shape[0]
        J = np.block([[A_el.toarray() / step.h ** 2, -Nm.T], [Nm, np.zeros((m, m))]])
        dx = np.linalg.solve(J, -F)
        q = q + dx[:N].reshape(-1, 3)
        lam = lam + dx[N:]
    return q, lam


def constrained_adjoint(step: Step, q_star, q_prev, dL_dq, dL_dv=None, Nm=None, with_multiplier=False):
    """z* of the equality-constrained step at its solution q_star (see the module docstring).
    With ``with_multiplier`` also w_l, which is dL/dd: the constraint targets d enter the KKT
    residual only as -d in its second block, so dL/dd = [b; 0]^T J^{-1} [0; I] = w_l."""
    free = _free(step)
    if Nm is None:
        Nm = _normals(step)
    m = Nm.shape[0]
    empty = np.zeros(0)
    A_el, _ = free.adjoint_matrix(State(q_star, empty, empty), q_prev)
    J = np.block([[A_el.toarray() / step.h ** 2, -Nm.T], [Nm, np.zeros((m, m))]])
    b = np.asarray(dL_dq, float).reshape(-1)
    if dL_dv is not None:
        b = b + np.asarray(dL_dv, float).reshape(-1) / step.h
    w = np.linalg.solve(J.T, np.concatenate([b, np.zeros(m)]))
    z = w[:step.N].reshape(-1, 3) / step.h ** 2
    return (z, w[step.N:]) if with_multiplier else z
