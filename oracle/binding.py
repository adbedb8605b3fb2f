"""Bilateral binding constraints (Eq. binding) on single vertices (test infrastructure: oracle).

Binding b attaches vertex v_b to a target point d_b through a compliant spring, the paper's
bilateral residual with J_b = e_{v_b}^T (x) I_3 (a prescribed attachment):
    delta_b = q_{v_b} - d_b,    phi_b = delta_b + E_b lambda_b = 0,
so lambda_b = -(q_{v_b} - d_b) / E_b with the compliance E_b > 0 (E_b -> 0: a hard attachment).
The momentum residual carries -h^2 J_b^T lambda_b = h^2 (q_{v_b} - d_b) / E_b at v_b, and the
adjoint matrix the block h^2 J_b^T E_b^{-1} J_b = h^2 / E_b I_3 on v_b's diagonal (Eq.
differential_2).  With the adjoint solution z (Eq. compute_gradient and the right-hand sides of
Eq. differential_2 for d_b and E_b):
    dL/dd_b = h^2 z_{v_b} / E_b,
    dL/dE_b = -h^2 z_{v_b} . lambda_b / E_b = h^2 z_{v_b} . (q_{v_b} - d_b) / E_b^2.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp


@dataclass
class Bindings:
    vertex: np.ndarray      # [n_b] int
    compliance: np.ndarray  # [n_b] > 0
    target: np.ndarray      # [n_b, 3]

    def __post_init__(self):
        self.vertex = np.asarray(self.vertex, dtype=np.int64).reshape(-1)
        self.compliance = np.asarray(self.compliance, float).reshape(-1)
        self.target = np.asarray(self.target, float).reshape(-1, 3)
        if not (len(self.vertex) == len(self.compliance) == len(self.target)):
            raise ValueError("vertex, compliance and target must have one entry per binding")
        if np.any(self.compliance <= 0):
            raise ValueError("compliance must be positive")

    @property
    def n(self):
        return len(self.vertex)

    def multipliers(self, q):
        """lambda_b [n_b, 3]."""
        return -(np.asarray(q, float)[self.vertex] - self.target) / self.compliance[:, None]

    def residual_term(self, q, h, n_verts):
        """The bindings' part of R_q (before the 1/h^2 scaling) [3 n_v]."""
        out = np.zeros((n_verts, 3))
        np.add.at(out, self.vertex, -h * h * self.multipliers(q))
        return out.reshape(-1)

    def matrix_term(self, h, n_verts):
        """h^2 / E_b I_3 on each bound vertex's diagonal [3 n_v, 3 n_v]."""
        d = np.zeros((n_verts, 3))
        np.add.at(d, self.vertex, (h * h / self.compliance)[:, None] * np.ones(3))
        return sp.diags(d.reshape(-1))

    def gradients(self, q, z, h):
        zv = np.asarray(z, float).reshape(-1, 3)[self.vertex]
        E = self.compliance
        dq = np.asarray(q, float)[self.vertex] - self.target
        return dict(dL_dbinding_target=h * h * zv / E[:, None],
                    dL_dcompliance=h * h * np.sum(zv * dq, axis=1) / E ** 2)
