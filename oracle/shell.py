"""Triangle (shell) elements: the 2D formulation of App. B.1 (test infrastructure, oracle).

A triangle's deformation gradient is F = D_s D_m^{-1} with D_s = [x1 - x0, x2 - x0] (3 x 2) and D_m the
rest edges in the triangle's own plane (2 x 2), so F has rank 2 and the thin SVD applies
(U 3 x 2, V 2 x 2, sigma in R^2).  Everything else of the volumetric derivation carries over:
the prox p(F) minimises w/2 ||P - F||^2 + zeta(P) per unit area, the element weight is
w_i = 2 mu_i A_i tau (tau: the shell's thickness, our reading of the paper's per-element weight),
and the lumped mass is rho tau A_i / 3 per corner.

Written here from the plain definitions:

* Neo-Hookean: zeta(P) = mu/2 (||P||^2 - log det C - 2) + lambda/2 (log J)^2 with C = P^T P and
  log J = (1/2) log det C; the prox is a damped Newton minimisation over the 6 entries of P, and
      grad zeta        = mu (P - P^+T) + lambda log J P^+T,           P^+T = P C^{-1},
      d(grad zeta)[dP] = mu dP + (lambda log J - mu) dP^+T + lambda (P^+T : dP) P^+T,
      dP^+T            = dP C^{-1} - P C^{-1} (dP^T P + P^T dP) C^{-1};
  dp/dF, dp/dmu and dp/dlambda follow from the implicit function theorem on
  2 mu (P - F) + grad zeta(P) = 0, as in the volumetric oracle.
* ARAP and co-rotational: through the thin polar decomposition F = R S (R 3 x 2 with orthonormal
  columns, S = (F^T F)^{1/2} symmetric positive definite): p = R, and
  p = R [ (S + I) / 2 - c (tr S - 2) I ] with c = lambda / (2 (4 mu + 2 lambda)) (the 2D form of the
  co-rotational stationarity condition).  The differential: R^T dF = Omega S + dS (Omega skew)
  gives the same Sylvester equation as in 3D, and the part of dR out of R's plane is
  (I - R R^T) dF S^{-1}.

Isometric bending (Bergou, Wardetzky, Harmon, Zorin, Grinspun 2006, "A quadratic bending model for
inextensible surfaces"): per interior edge the constant stencil K of cotangent weights over the
edge's four vertices, Q_e = 3 / (A_1 + A_2) K K^T, and the energy 1/2 k_b sum_e x^T (Q_e (x) I_3) x.
Its Hessian is the constant k_b Q: it enters the elastic matrix A and no projection.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse as sp


def vec6(X):
    """Column stacking of [..., 3, 2] -> [..., 6]: vec(X)[r + 3k] = X[r, k]."""
    return np.swapaxes(X, -1, -2).reshape(X.shape[:-2] + (6,))


def unvec6(v):
    return np.swapaxes(v.reshape(v.shape[:-1] + (2, 3)), -1, -2)


class TriMesh:
    """Per-triangle rest operators of a triangle mesh, with the interface of the tet Mesh."""

    nF = 6

    def __init__(self, X, tris, thickness):
        self.X = np.asarray(X, float)
        self.tets = np.asarray(tris, np.int64)  # the element array (named as in Mesh)
        self.n_verts = self.X.shape[0]
        self.n_tets = self.tets.shape[0]
        self.thickness = float(thickness)
        e1 = self.X[self.tets[:, 1]] - self.X[self.tets[:, 0]]
        e2 = self.X[self.tets[:, 2]] - self.X[self.tets[:, 0]]
        nrm = np.cross(e1, e2)
        area2 = np.linalg.norm(nrm, axis=1)
        if np.any(area2 <= 0):
            raise ValueError("mesh has degenerate triangles")
        a1 = e1 / np.linalg.norm(e1, axis=1)[:, None]
        a2 = np.cross(nrm / area2[:, None], a1)
        Dm = np.stack([np.stack([np.sum(a1 * e1, 1), np.sum(a1 * e2, 1)], 1),
                       np.stack([np.sum(a2 * e1, 1), np.sum(a2 * e2, 1)], 1)], 1)  # [n, 2, 2]
        self.B = np.linalg.inv(Dm)
        self.area = 0.5 * area2
        self.vol = self.area * self.thickness
        g = np.zeros((self.n_tets, 3, 2))
        g[:, 1:, :] = self.B
        g[:, 0, :] = -self.B.sum(axis=1)
        self.g = g
        G = np.zeros((self.n_tets, 6, 9))
        for a in range(3):
            for k in range(2):
                for r in range(3):
                    G[:, r + 3 * k, 3 * a + r] = g[:, a, k]
        self.G = G
        self.dofs = (3 * self.tets[:, :, None] + np.arange(3)[None, None, :]).reshape(self.n_tets, 9)

    vec = staticmethod(vec6)
    unvec = staticmethod(unvec6)

    def F(self, q):
        return unvec6(np.einsum("tij,tj->ti", self.G, q.reshape(-1)[self.dofs]))

    def Gx(self, x):
        return np.einsum("tij,tj->ti", self.G, x.reshape(-1)[self.dofs])

    def min_jacobian(self, F):
        """The smallest sqrt(det F^T F) (zero for a collapsed triangle)."""
        return float(np.sqrt(np.maximum(np.linalg.det(np.swapaxes(F, 1, 2) @ F), 0.0)).min())

    def lumped_mass(self, density):
        m = np.zeros(self.n_verts)
        np.add.at(m, self.tets.ravel(), np.repeat(density * self.vol / 3.0, 3))
        return m

    def scatter_blocks(self, blocks):
        rows = np.repeat(self.dofs, 9, axis=1).ravel()
        cols = np.tile(self.dofs, (1, 9)).ravel()
        N = 3 * self.n_verts
        return sp.coo_matrix((blocks.ravel(), (rows, cols)), shape=(N, N)).tocsr()

    def scatter_vectors(self, vecs9):
        out = np.zeros(3 * self.n_verts)
        np.add.at(out, self.dofs.ravel(), vecs9.ravel())
        return out

    # ---- isometric bending ------------------------------------------------------------
    def bending_stencils(self):
        """[(i0, i1, i2, i3), K (4,), A1 + A2] per interior edge (i0, i1) with opposite vertices i2, i3."""
        opp = {}
        for t, (a, b, c) in enumerate(self.tets):
            for u, v, w in ((a, b, c), (b, c, a), (c, a, b)):
                opp.setdefault((min(u, v), max(u, v)), []).append(w)
        out = []
        X = self.X
        cot = lambda p, q: (p @ q) / np.linalg.norm(np.cross(p, q))  # noqa: E731
        for (i0, i1), ws in sorted(opp.items()):
            if len(ws) != 2:
                continue
            i2, i3 = ws
            e0, e1, e2 = X[i1] - X[i0], X[i2] - X[i0], X[i3] - X[i0]
            e3, e4 = X[i2] - X[i1], X[i3] - X[i1]
            c01, c02 = cot(e0, e1), cot(e0, e2)
            c03, c04 = cot(-e0, e3), cot(-e0, e4)
            K = np.array([c03 + c04, c01 + c02, -c01 - c03, -c02 - c04])
            A = 0.5 * (np.linalg.norm(np.cross(e0, e1)) + np.linalg.norm(np.cross(e0, e2)))
            out.append(((i0, i1, i2, i3), K, A))
        return out

    def bending_matrix(self):
        """Q = sum_e 3/(A_1 + A_2) (K K^T) (x) I_3, sparse [3 n_v, 3 n_v] (the energy is 1/2 k_b q^T Q q)."""
        rows, cols, vals = [], [], []
        for idx, K, A in self.bending_stencils():
            Qe = 3.0 / A * np.outer(K, K)
            for a in range(4):
                for b in range(4):
                    for r in range(3):
                        rows.append(3 * idx[a] + r)
                        cols.append(3 * idx[b] + r)
                        vals.append(Qe[a, b])
        N = 3 * self.n_verts
        return sp.coo_matrix((vals, (rows, cols)), shape=(N, N)).tocsr()


# ---- projections of 3 x 2 deformation gradients --------------------------------------------
NEO_HOOKEAN, COROTATIONAL, ARAP = "neo_hookean", "corotational", "arap"


class DegenerateElement(ValueError):
    pass


def _pinvT(P):
    """P C^{-1}, C = P^T P (the transposed pseudo-inverse of a rank-2 3 x 2 matrix), and C^{-1}."""
    Ci = np.linalg.inv(np.swapaxes(P, -1, -2) @ P)
    return P @ Ci, Ci


def _logJ(P):
    return 0.5 * np.log(np.linalg.det(np.swapaxes(P, -1, -2) @ P))


def nh_zeta(P, mu, lam):
    C = np.swapaxes(P, -1, -2) @ P
    ld = np.log(np.linalg.det(C))
    return 0.5 * mu * (np.sum(P * P, axis=(-1, -2)) - ld - 2.0) + 0.5 * lam * (0.5 * ld) ** 2


def nh_grad(P, mu, lam):
    PT, _ = _pinvT(P)
    mu_ = np.asarray(mu)[..., None, None]
    lam_ = np.asarray(lam)[..., None, None]
    return mu_ * (P - PT) + lam_ * _logJ(P)[..., None, None] * PT


def nh_hess(P, mu, lam):
    """6 x 6 Hessian of zeta in the vec6 basis, [..., 6, 6]."""
    PT, Ci = _pinvT(P)
    lJ = _logJ(P)
    mu = np.asarray(mu, float)
    lam = np.asarray(lam, float)
    H = np.zeros(P.shape[:-2] + (6, 6))
    for m in range(6):
        e = np.zeros(6)
        e[m] = 1.0
        dP = unvec6(np.broadcast_to(e, P.shape[:-2] + (6,)))
        dC = np.swapaxes(dP, -1, -2) @ P + np.swapaxes(P, -1, -2) @ dP
        dPT = dP @ Ci - P @ Ci @ dC @ Ci
        term = (mu[..., None, None] * dP + (lam * lJ - mu)[..., None, None] * dPT
                + lam[..., None, None] * np.sum(PT * dP, axis=(-1, -2))[..., None, None] * PT)
        H[..., :, m] = vec6(term)
    return H


def nh_prox(F, mu, lam, tol=1e-14, max_iter=100):
    """argmin_P mu ||P - F||^2 + zeta(P) for F [n, 3, 2] by damped Newton over the 6 entries of P."""
    F = np.asarray(F, float)
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,)).copy()
    lam = np.broadcast_to(np.asarray(lam, float), (n,)).copy()
    if np.any(np.linalg.det(np.swapaxes(F, 1, 2) @ F) <= 0):
        raise DegenerateElement("a collapsed triangle (rank F < 2)")
    P = F.copy()

    def objective(Q):
        return mu * np.sum((Q - F) ** 2, axis=(1, 2)) + nh_zeta(Q, mu, lam)

    for _ in range(max_iter):
        g = 2.0 * mu[:, None, None] * (P - F) + nh_grad(P, mu, lam)
        gn = np.max(np.abs(g), axis=(1, 2)) / mu
        if np.all(gn <= tol):
            break
        H = 2.0 * mu[:, None, None] * np.eye(6) + nh_hess(P, mu, lam)
        step = -unvec6(np.linalg.solve(H, vec6(g)[..., None])[..., 0])
        f0 = objective(P)
        t = np.ones(n)
        active = gn > tol
        for _ in range(60):
            Pt = P + t[:, None, None] * step
            ok = np.linalg.det(np.swapaxes(Pt, 1, 2) @ Pt) > 0
            ft = np.where(ok, objective(np.where(ok[:, None, None], Pt, P)), np.inf)
            good = ok & ((ft <= f0 + 1e-4 * t * np.sum(vec6(g) * vec6(step), axis=1)) | (gn < 1e-6))
            if np.all(good | ~active):
                break
            t = np.where(good | ~active, t, 0.5 * t)
        P = np.where(active[:, None, None], P + t[:, None, None] * step, P)
    return P


def nh_prox_derivatives(F, P, mu, lam):
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,))
    lam = np.broadcast_to(np.asarray(lam, float), (n,))
    H = 2.0 * mu[:, None, None] * np.eye(6) + nh_hess(P, mu, lam)
    Hinv = np.linalg.inv(H)
    PT, _ = _pinvT(P)
    g_mu = 2.0 * (P - F) + P - PT
    g_lam = _logJ(P)[:, None, None] * PT
    return (2.0 * mu[:, None, None] * Hinv, -unvec6(np.einsum("nij,nj->ni", Hinv, vec6(g_mu))),
            -unvec6(np.einsum("nij,nj->ni", Hinv, vec6(g_lam))))


def thin_polar(F):
    """(R, S, Q, s): F = R S, R [n, 3, 2] with orthonormal columns, S = Q diag(s) Q^T [n, 2, 2]."""
    e, Q = np.linalg.eigh(np.swapaxes(F, 1, 2) @ F)
    if np.any(e <= 0):
        raise DegenerateElement("a collapsed triangle (rank F < 2)")
    s = np.sqrt(e)
    S = (Q * s[:, None, :]) @ np.swapaxes(Q, 1, 2)
    R = F @ ((Q / s[:, None, :]) @ np.swapaxes(Q, 1, 2))
    return R, S, Q, s


def thin_polar_differential(R, S, Q, s, dF):
    """(dR, dS) of F = R S along dF [n, 3, 2]: the in-plane part from the Sylvester equation
    S Omega + Omega S = R^T dF - dF^T R (solved in S's eigenbasis), the out-of-plane part
    (I - R R^T) dF S^{-1}."""
    Rt = np.swapaxes(R, 1, 2)
    X = Rt @ dF - np.swapaxes(dF, 1, 2) @ R
    Qt = np.swapaxes(Q, 1, 2)
    Om = Q @ ((Qt @ X @ Q) / (s[:, :, None] + s[:, None, :])) @ Qt
    dS = Rt @ dF - Om @ S
    Sinv = (Q / s[:, None, :]) @ Qt
    out = dF - R @ (Rt @ dF)
    return R @ Om + out @ Sinv, dS


def corot_c2(mu, lam):
    return lam / (2.0 * (4.0 * mu + 2.0 * lam))


def prox(model, F, mu, lam):
    """p(F) for F [n, 3, 2]; model one name or one per item."""
    F = np.asarray(F, float)
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,))
    lam = np.broadcast_to(np.asarray(lam, float), (n,))
    if not isinstance(model, str):
        model = np.asarray(model)
        P = np.zeros_like(F)
        for m in (NEO_HOOKEAN, COROTATIONAL, ARAP):
            idx = np.nonzero(model == m)[0]
            if len(idx):
                P[idx] = prox(m, F[idx], mu[idx], lam[idx])
        return P
    if model == NEO_HOOKEAN:
        return nh_prox(F, mu, lam)
    R, S, _, _ = thin_polar(F)
    if model == ARAP:
        return R
    if model != COROTATIONAL:
        raise ValueError(f"unknown model {model!r}")
    c = corot_c2(mu, lam)[:, None, None]
    I2 = np.eye(2)
    return R @ (0.5 * (S + I2) - c * (np.trace(S, axis1=1, axis2=2)[:, None, None] - 2.0) * I2)


def prox_derivatives(model, F, P, mu, lam):
    """dP/dF [n, 6, 6] (vec6 basis), dP/dmu [n, 3, 2], dP/dlam [n, 3, 2] at P = prox(model, F)."""
    F = np.asarray(F, float)
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,))
    lam = np.broadcast_to(np.asarray(lam, float), (n,))
    if not isinstance(model, str):
        model = np.asarray(model)
        Jp, dmu, dlam = np.zeros((n, 6, 6)), np.zeros((n, 3, 2)), np.zeros((n, 3, 2))
        for m in (NEO_HOOKEAN, COROTATIONAL, ARAP):
            idx = np.nonzero(model == m)[0]
            if len(idx):
                Jp[idx], dmu[idx], dlam[idx] = prox_derivatives(m, F[idx], None if P is None else P[idx],
                                                                mu[idx], lam[idx])
        return Jp, dmu, dlam
    if model == NEO_HOOKEAN:
        return nh_prox_derivatives(F, P, mu, lam)
    R, S, Q, s = thin_polar(F)
    I2 = np.eye(2)
    trS = np.trace(S, axis1=1, axis2=2)[:, None, None]
    c = corot_c2(mu, lam)[:, None, None]
    K = 0.5 * (S + I2) - c * (trS - 2.0) * I2
    Jp = np.zeros((n, 6, 6))
    for m in range(6):
        e = np.zeros(6)
        e[m] = 1.0
        dR, dS = thin_polar_differential(R, S, Q, s, np.broadcast_to(unvec6(e), F.shape))
        if model == ARAP:
            dP = dR
        else:
            dP = dR @ K + R @ (0.5 * dS - c * np.trace(dS, axis1=1, axis2=2)[:, None, None] * I2)
        Jp[:, :, m] = vec6(dP)
    dmu = np.zeros((n, 3, 2))
    dlam = np.zeros((n, 3, 2))
    if model == COROTATIONAL:
        den = ((4.0 * mu + 2.0 * lam) ** 2)[:, None, None]
        dmu = R * ((trS - 2.0) * 2.0 * lam[:, None, None] / den)
        dlam = -R * ((trS - 2.0) * 2.0 * mu[:, None, None] / den)
    return Jp, dmu, dlam
