"""Bilateral binding constraints (Eq. binding) on points of the mesh (test infrastructure: oracle).

Binding b attaches a point of the mesh, J_b q = sum_k w_bk q_{v_bk} (one vertex with weight 1, or
a point inside a tet given by its barycentric weights), to a target point d_b through a
compliant spring, the paper's bilateral residual with J_b = w_b^T (x) I_3:
    delta_b = J_b q - d_b,    phi_b = delta_b + E_b lambda_b = 0,
so lambda_b = -(J_b q - d_b) / E_b with the compliance E_b > 0 (E_b -> 0: a hard attachment).
The momentum residual carries -h^2 J_b^T lambda_b, i.e. h^2 w_bk (J_b q - d_b) / E_b at each
v_bk, and the adjoint matrix the blocks h^2 J_b^T E_b^{-1} J_b = h^2 w_bk w_bl / E_b I_3 at
(v_bk, v_bl) (Eq. differential_2).  With the adjoint solution z (Eq. compute_gradient and the
right-hand sides of Eq. differential_2 for d_b and E_b):
    dL/dd_b = h^2 (J_b z) / E_b,
    dL/dE_b = -h^2 (J_b z) . lambda_b / E_b = h^2 (J_b z) . (J_b q - d_b) / E_b^2.
"""
from __future__ import annotations

from dataclasses import dataclass
from typing import Optional

import numpy as np
import scipy.sparse as sp


@dataclass
class Bindings:
    vertex: np.ndarray                   # [n_b] int, or [n_b, k] for points spanned by k vertices
    compliance: np.ndarray               # [n_b] > 0
    target: np.ndarray                   # [n_b, 3]
    weight: Optional[np.ndarray] = None  # [n_b, k] (None: one vertex per binding, weight 1)

    def __post_init__(self):
        self.vertex = np.asarray(self.vertex, dtype=np.int64)
        n = self.vertex.shape[0]
        # the spanning vertices and weights as [n_b, k] whatever the form given
        self.vk = self.vertex.reshape(n, -1)
        self.wk = (np.ones(self.vk.shape) if self.weight is None else np.asarray(self.weight, float).reshape(n, -1))
        self.compliance = np.asarray(self.compliance, float).reshape(-1)
        self.target = np.asarray(self.target, float).reshape(-1, 3)
        if not (self.wk.shape == self.vk.shape and len(self.compliance) == n and len(self.target) == n):
            raise ValueError("vertex, weight, compliance and target must have one entry per binding")
        if np.any(self.compliance <= 0):
            raise ValueError("compliance must be positive")

    @property
    def n(self):
        return self.vk.shape[0]

    def point(self, x):
        """J_b x for every binding [n_b, 3] (x [n_v, 3])."""
        x = np.asarray(x, float).reshape(-1, 3)
        return np.einsum("bk,bkj->bj", self.wk, x[self.vk])

    def multipliers(self, q):
        """lambda_b [n_b, 3]."""
        return -(self.point(q) - self.target) / self.compliance[:, None]

    def residual_term(self, q, h, n_verts):
        """The bindings' part of R_q (before the 1/h^2 scaling) [3 n_v]."""
        out = np.zeros((n_verts, 3))
        f = -h * h * self.multipliers(q)
        for k in range(self.vk.shape[1]):
            np.add.at(out, self.vk[:, k], self.wk[:, k, None] * f)
        return out.reshape(-1)

    def matrix_term(self, h, n_verts):
        """h^2 / E_b w_bk w_bl I_3 at (v_bk, v_bl) [3 n_v, 3 n_v]."""
        rows, cols, vals = [], [], []
        kk = self.vk.shape[1]
        for b in range(self.n):
            c = h * h / self.compliance[b]
            for k in range(kk):
                for m in range(kk):
                    for r in range(3):
                        rows.append(3 * self.vk[b, k] + r)
                        cols.append(3 * self.vk[b, m] + r)
                        vals.append(c * self.wk[b, k] * self.wk[b, m])
        N = 3 * n_verts
        return sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()

    def rows(self, n_verts):
        """The constraint rows J_b stacked [3 n_b, 3 n_v] (hard attachments J q = d)."""
        Nm = np.zeros((3 * self.n, 3 * n_verts))
        for b in range(self.n):
            for k in range(self.vk.shape[1]):
                v = self.vk[b, k]
                Nm[3 * b:3 * b + 3, 3 * v:3 * v + 3] += self.wk[b, k] * np.eye(3)
        return Nm

    def gradients(self, q, z, h):
        Jz = self.point(np.asarray(z, float).reshape(-1, 3))
        E = self.compliance
        dq = self.point(q) - self.target
        return dict(dL_dbinding_target=h * h * Jz / E[:, None],
                    dL_dcompliance=h * h * np.sum(Jz * dq, axis=1) / E ** 2)
