"""Discrete model: per-tet operators, lumped mass, Lame parameters, the elastic matrix A.

Test infrastructure (oracle); see the package docstring.

Conventions (Sec. 3.1-3.3, App. B.0):
* DOF order: q[3 v + r] is coordinate r of vertex v.
* vec() stacks columns: vec(X)[r + 3k] = X[r, k].
* D_m = [X1-X0, X2-X0, X3-X0], B = D_m^{-1}, F = D_s B, V = |det D_m| / 6.
* G_i (9 x 12) maps the tet's 12 local DOFs to vec(F):  G_i[r + 3k, 3a + s] = delta_rs g_a[k],
  with g_a = row (a-1) of B for a = 1..3 and g_0 = -(g_1 + g_2 + g_3).
* Lumped mass m_v = rho * sum_{i ∋ v} V_i / 4.  w_i = 2 mu_i V_i and zeta_i = V_i zeta (the
  paper states w = 2 mu per unit volume, App. B.2; the V_i factor is our reading).
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def vec(X):
    """Column-stacking vectorisation of [..., 3, 3] -> [..., 9]."""
    return np.swapaxes(X, -1, -2).reshape(X.shape[:-2] + (9,))


def unvec(v):
    """Inverse of vec: [..., 9] -> [..., 3, 3]."""
    return np.swapaxes(v.reshape(v.shape[:-1] + (3, 3)), -1, -2)


def lame(E, nu):
    """mu, lambda from Young's modulus and Poisson's ratio (App. B.3)."""
    E = np.asarray(E, float)
    nu = np.asarray(nu, float)
    return E / (2.0 * (1.0 + nu)), E * nu / ((1.0 + nu) * (1.0 - 2.0 * nu))


def lame_derivatives(E, nu):
    """d(mu, lambda)/d(E, nu) as four arrays: dmu_dE, dlam_dE, dmu_dnu, dlam_dnu."""
    E = np.asarray(E, float)
    nu = np.asarray(nu, float)
    dmu_dE = 1.0 / (2.0 * (1.0 + nu))
    dlam_dE = nu / ((1.0 + nu) * (1.0 - 2.0 * nu))
    dmu_dnu = -E / (2.0 * (1.0 + nu) ** 2)
    dlam_dnu = E * (1.0 + 2.0 * nu ** 2) / ((1.0 + nu) * (1.0 - 2.0 * nu)) ** 2
    return dmu_dE, dlam_dE, dmu_dnu, dlam_dnu


class Mesh:
    """Per-tet rest operators of a tet mesh (float64)."""

    nF = 9  # entries of vec(F)

    def __init__(self, X, tets):
        self.X = np.asarray(X, float)
        self.tets = np.asarray(tets, np.int64)
        self.n_verts = self.X.shape[0]
        self.n_tets = self.tets.shape[0]
        Dm = np.swapaxes(self.X[self.tets[:, 1:]] - self.X[self.tets[:, [0]]], 1, 2)  # columns = edges
        det = np.linalg.det(Dm)
        if np.any(det <= 0):
            raise ValueError("mesh has inverted or degenerate tets")
        self.B = np.linalg.inv(Dm)
        self.vol = det / 6.0
        g = np.zeros((self.n_tets, 4, 3))
        g[:, 1:, :] = self.B
        g[:, 0, :] = -self.B.sum(axis=1)
        self.g = g
        G = np.zeros((self.n_tets, 9, 12))
        for a in range(4):
            for k in range(3):
                for r in range(3):
                    G[:, r + 3 * k, 3 * a + r] = g[:, a, k]
        self.G = G
        # global DOF ids of each tet's 12 local DOFs
        self.dofs = (3 * self.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(self.n_tets, 12)

    vec = staticmethod(vec)
    unvec = staticmethod(unvec)

    def min_jacobian(self, F):
        """The smallest det F (<= 0: some tet inverted)."""
        return float(np.linalg.det(F).min())

    def F(self, q):
        """Deformation gradients [n_t, 3, 3] of positions q [n_v, 3]."""
        return unvec(np.einsum("tij,tj->ti", self.G, q.reshape(-1)[self.dofs]))

    def Gx(self, x):
        """vec(G_i x) [n_t, 9] for a DOF vector x [3 n_v]."""
        return np.einsum("tij,tj->ti", self.G, x.reshape(-1)[self.dofs])

    def lumped_mass(self, density):
        m = np.zeros(self.n_verts)
        np.add.at(m, self.tets.ravel(), np.repeat(density * self.vol / 4.0, 4))
        return m

    def scatter_blocks(self, blocks):
        """Sparse 3n x 3n matrix from per-tet 12x12 blocks [n_t, 12, 12]."""
        rows = np.repeat(self.dofs, 12, axis=1).ravel()
        cols = np.tile(self.dofs, (1, 12)).ravel()
        N = 3 * self.n_verts
        return sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(N, N)).tocsr()

    def scatter_vectors(self, vecs12):
        """DOF vector [3n] from per-tet 12-vectors [n_t, 12] (summed)."""
        out = np.zeros(3 * self.n_verts)
        np.add.at(out, self.dofs.ravel(), vecs12.ravel())
        return out


def elastic_matrix(mesh: Mesh, mass, mu, h):
    """A = M + h^2 sum_i w_i G_i^T G_i  (Eq. dynamics), w_i = 2 mu_i V_i."""
    w = 2.0 * np.asarray(mu) * mesh.vol
    blocks = h * h * w[:, None, None] * np.einsum("tki,tkj->tij", mesh.G, mesh.G)
    return sp.diags(np.repeat(mass, 3)) + mesh.scatter_blocks(blocks)
