"""Woodbury form of the contact-regime preconditioner, dense, for tiny meshes.

Test infrastructure (oracle); see the package docstring.

Eq. (woodbury_formula) inverts K pointwise; K_c has exact zeros (mu = 0) and near-zero
entries (sliding, separating), so the algebraically identical form without K^{-1} is used:
    (A + h^2 J^T K J)^{-1} = A^{-1} - h^2 A^{-1} J^T (I + h^2 K D)^{-1} K J A^{-1},
    D = J A^{-1} J^T   (the Delassus operator).
For the transposed system the same holds with K replaced by K^T.
"""
from __future__ import annotations

import numpy as np


def contact_jacobian_matrix(n_verts, vertex, frame):
    """Dense J [3 n_c, 3 n_v]: rows of contact c are its frame rows acting on vertex v_c."""
    nc = len(vertex)
    J = np.zeros((3 * nc, 3 * n_verts))
    for c in range(nc):
        v = vertex[c]
        J[3 * c:3 * c + 3, 3 * v:3 * v + 3] = frame[c]
    return J


def woodbury_apply(A, J, Kblk, h, r):
    """(A + h^2 J^T blockdiag(Kblk) J)^{-1} r by the stable Woodbury form (dense)."""
    A = np.asarray(A.todense()) if hasattr(A, "todense") else np.asarray(A)
    nc = Kblk.shape[0]
    K = np.zeros((3 * nc, 3 * nc))
    for c in range(nc):
        K[3 * c:3 * c + 3, 3 * c:3 * c + 3] = Kblk[c]
    u = np.linalg.solve(A, r)
    D = J @ np.linalg.solve(A, J.T)
    Cap = np.eye(3 * nc) + h * h * K @ D
    t = np.linalg.solve(Cap, K @ (J @ u))
    return u - h * h * np.linalg.solve(A, J.T @ t)
