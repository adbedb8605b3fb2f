"""Neo-Hookean local projection (prox) and its derivatives, from their plain definitions.

Test infrastructure (oracle); see the package docstring.

Per unit volume (the V_i factors cancel, w = 2 mu):
    p(F) = argmin_P  mu ||P - F||^2 + zeta(P),                                (Eq. internal)
    zeta(P) = mu/2 (||P||^2 - log det(P^T P) - 3) + lambda/8 (log det(P^T P))^2   (App. B.2)
            = mu/2 (||P||^2 - 2 log J - 3) + lambda/2 (log J)^2,  J = det P.
    grad zeta(P)          = mu (P - P^{-T}) + lambda log J P^{-T}
    grad^2 zeta(P)[dP]    = mu dP + (mu - lambda log J) P^{-T} dP^T P^{-T} + lambda (P^{-T}:dP) P^{-T}

The minimiser is found by damped Newton over the 9 entries of P (no SVD).  Its derivatives
follow from the implicit function theorem on the stationarity condition
    g(P; F, mu, lambda) = 2 mu (P - F) + grad zeta(P) = 0:
    dp/dF      = 2 mu H^{-1}                          (= (I + grad^2 zeta / w)^{-1}, Eq. pd_expanded)
    dp/dmu     = -H^{-1} [2 (P - F) + P - P^{-T}]     (w = 2 mu varies with mu, App. B.3)
    dp/dlambda = -H^{-1} [log J P^{-T}]
with H = 2 mu I + grad^2 zeta(P) the 9x9 Hessian.
"""
from __future__ import annotations

import numpy as np

from .model import unvec, vec


class InvertedElement(ValueError):
    pass


def zeta(P, mu, lam):
    J = np.linalg.det(P)
    lJ = np.log(J)
    return 0.5 * mu * (np.sum(P * P, axis=(-1, -2)) - 2.0 * lJ - 3.0) + 0.5 * lam * lJ ** 2


def grad_zeta(P, mu, lam):
    J = np.linalg.det(P)
    PiT = np.swapaxes(np.linalg.inv(P), -1, -2)
    mu_ = np.asarray(mu)[..., None, None]
    lam_ = np.asarray(lam)[..., None, None]
    return mu_ * (P - PiT) + lam_ * np.log(J)[..., None, None] * PiT


def hess_zeta(P, mu, lam):
    """9x9 Hessian of zeta in the vec() basis, [..., 9, 9]."""
    J = np.linalg.det(P)
    PiT = np.swapaxes(np.linalg.inv(P), -1, -2)
    c = np.asarray(mu) - np.asarray(lam) * np.log(J)
    H = np.zeros(P.shape[:-2] + (9, 9))
    for m in range(9):
        e = np.zeros(9)
        e[m] = 1.0
        dP = unvec(np.broadcast_to(e, P.shape[:-2] + (9,)))
        term = (np.asarray(mu)[..., None, None] * dP
                + c[..., None, None] * (PiT @ np.swapaxes(dP, -1, -2) @ PiT)
                + np.asarray(lam)[..., None, None] * np.sum(PiT * dP, axis=(-1, -2))[..., None, None] * PiT)
        H[..., :, m] = vec(term)
    return H


def prox_objective(P, F, mu, lam):
    return mu * np.sum((P - F) ** 2, axis=(-1, -2)) + zeta(P, mu, lam)


def prox(F, mu, lam, tol=1e-14, max_iter=100):
    """p(F) for a batch of F [n, 3, 3] with per-item mu, lam [n].  Returns P [n, 3, 3].

    Raises InvertedElement if det F <= 0 (the Neo-Hookean energy needs J > 0).
    """
    F = np.asarray(F, float)
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,)).copy()
    lam = np.broadcast_to(np.asarray(lam, float), (n,)).copy()
    if np.any(np.linalg.det(F) <= 0):
        raise InvertedElement("det F <= 0")
    P = F.copy()
    for _ in range(max_iter):
        g = 2.0 * mu[:, None, None] * (P - F) + grad_zeta(P, mu, lam)
        gn = np.max(np.abs(g), axis=(1, 2)) / mu
        if np.all(gn <= tol):
            break
        H = 2.0 * mu[:, None, None] * np.eye(9) + hess_zeta(P, mu, lam)
        step = -unvec(np.linalg.solve(H, vec(g)[..., None])[..., 0])
        f0 = prox_objective(P, F, mu, lam)
        t = np.ones(n)
        active = gn > tol
        for _ in range(60):
            Pt = P + t[:, None, None] * step
            ok = np.linalg.det(Pt) > 0
            ft = np.where(ok, prox_objective(np.where(ok[:, None, None], Pt, P), F, mu, lam), np.inf)
            # accept full steps once close (objective differences drown in rounding there)
            good = ok & ((ft <= f0 + 1e-4 * t * np.sum(vec(g) * vec(step), axis=1)) | (gn < 1e-6))
            if np.all(good | ~active):
                break
            t = np.where(good | ~active, t, 0.5 * t)
        P = np.where(active[:, None, None], P + t[:, None, None] * step, P)
    return P


def prox_derivatives(F, P, mu, lam):
    """Jacobians at a converged prox: dP/dF [n,9,9], dP/dmu [n,3,3], dP/dlam [n,3,3]."""
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,))
    lam = np.broadcast_to(np.asarray(lam, float), (n,))
    H = 2.0 * mu[:, None, None] * np.eye(9) + hess_zeta(P, mu, lam)
    Hinv = np.linalg.inv(H)
    Jp = 2.0 * mu[:, None, None] * Hinv
    PiT = np.swapaxes(np.linalg.inv(P), -1, -2)
    logJ = np.log(np.linalg.det(P))
    g_mu = 2.0 * (P - F) + P - PiT
    g_lam = logJ[:, None, None] * PiT
    dP_dmu = -unvec(np.einsum("nij,nj->ni", Hinv, vec(g_mu)))
    dP_dlam = -unvec(np.einsum("nij,nj->ni", Hinv, vec(g_lam)))
    return Jp, dP_dmu, dP_dlam
