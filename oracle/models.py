"""Co-rotational and ARAP local projections and their derivatives (test infrastructure: oracle).

App. B.2 names three isotropic models that share the SVD projection Jacobian of Sec. 4.3 and
differ only in theta(sigma) and W = dtheta/dsigma.  The Neo-Hookean prox is in ``prox``; this
module writes out the other two from their definitions, through the polar decomposition
F = R S (R a rotation, S symmetric positive definite), not through the SVD formulas of App. B:

* ARAP keeps only the rotation: p(F) = R.  The energy is w/2 ||F - R||^2 with w = 2 mu, so
  mu enters only through the weight: dp/dmu = dp/dlambda = 0.
* Co-rotational: zeta(theta) = mu ||theta - 1||^2 + lambda/2 (sum_i (theta_i - 1))^2 on the
  singular values, w = 2 mu.  Its stationarity condition is linear in theta,
      4 mu (theta - 1) + lambda tr(theta - 1) 1 = 2 mu (sigma - 1),
  so theta - 1 = W (sigma - 1) with the constant W = 1/2 I - c 1 1^T, c = lambda / (2 (4 mu + 3 lambda)).
  Since S = V diag(sigma) V^T and R = U V^T, the projection is, without any SVD,
      p(F) = R [ (S + I) / 2 - c (tr S - 3) I ].
  Its parameter derivatives act only through c:
      dp/dmu = R (tr S - 3) * 2 lambda / (4 mu + 3 lambda)^2,
      dp/dlambda = -R (tr S - 3) * 2 mu / (4 mu + 3 lambda)^2.

dp/dF comes from the differential of the polar decomposition.  With dR = R Omega (Omega skew)
and dS symmetric, R^T dF = Omega S + dS; its antisymmetric part gives the Sylvester equation
    S Omega + Omega S = R^T dF - dF^T R,
after which dS = R^T dF - Omega S.  ``polar_differential`` solves it with a library Sylvester
solver; the batched path used by the step solves it in the eigenbasis of S = Q diag(s) Q^T,
where it decouples: (Q^T Omega Q)_ij = (Q^T X Q)_ij / (s_i + s_j).  The two are pinned equal.

Both models need det F > 0 here (the polar rotation of an inverted F is a reflection); the
kernels take the same rule for every model.
"""
from __future__ import annotations

import numpy as np
from scipy.linalg import polar, solve_sylvester

from .model import unvec, vec
from . import prox as _nh
from .prox import InvertedElement

NEO_HOOKEAN, COROTATIONAL, ARAP = "neo_hookean", "corotational", "arap"
MODELS = (NEO_HOOKEAN, COROTATIONAL, ARAP)


def polar_one(F):
    """(R, S) of one F by the library polar decomposition."""
    if np.linalg.det(F) <= 0:
        raise InvertedElement("det F <= 0")
    R, S = polar(F, side="right")
    return R, 0.5 * (S + S.T)


def polar_differential(R, S, dF):
    """(dR, dS) of F = R S along dF."""
    X = R.T @ dF - dF.T @ R
    Om = solve_sylvester(S, S, X)
    Om = 0.5 * (Om - Om.T)
    return R @ Om, R.T @ dF - Om @ S


def polar_batch(F):
    """(R, S, Q, s) for F [n, 3, 3]: F = R S with S = Q diag(s) Q^T from the symmetric
    eigendecomposition of F^T F (s = sqrt of its eigenvalues)."""
    if np.any(np.linalg.det(F) <= 0):
        raise InvertedElement("det F <= 0")
    e, Q = np.linalg.eigh(np.swapaxes(F, 1, 2) @ F)
    s = np.sqrt(e)
    S = (Q * s[:, None, :]) @ np.swapaxes(Q, 1, 2)
    R = F @ ((Q / s[:, None, :]) @ np.swapaxes(Q, 1, 2))
    return R, S, Q, s


def polar_differential_batch(R, S, Q, s, dF):
    """(dR, dS) of F = R S along dF [n, 3, 3] (the eigenbasis solution of the Sylvester equation)."""
    Rt = np.swapaxes(R, 1, 2)
    X = Rt @ dF - np.swapaxes(dF, 1, 2) @ R
    Qt = np.swapaxes(Q, 1, 2)
    Om = Q @ ((Qt @ X @ Q) / (s[:, :, None] + s[:, None, :])) @ Qt
    return R @ Om, Rt @ dF - Om @ S


def corot_c(mu, lam):
    return lam / (2.0 * (4.0 * mu + 3.0 * lam))


def zeta_corotational(P, mu, lam):
    """zeta of the co-rotational model as a function of P, through P's polar factor S_P
    (its eigenvalues are P's singular values): mu ||S_P - I||^2 + lambda/2 (tr S_P - 3)^2."""
    _, S = polar_one(P)
    return mu * np.sum((S - np.eye(3)) ** 2) + 0.5 * lam * (np.trace(S) - 3.0) ** 2


def by_model(model, n):
    """[(model name, item indices)] for one name or a per-item sequence of names."""
    if isinstance(model, str):
        if model not in MODELS:
            raise ValueError(f"unknown model {model!r}")
        return [(model, np.arange(n))]
    model = np.asarray(model)
    if model.shape != (n,) or not set(model.tolist()) <= set(MODELS):
        raise ValueError("per-item models must be names from MODELS, one per item")
    return [(m, np.nonzero(model == m)[0]) for m in MODELS if np.any(model == m)]


def prox(model, F, mu, lam):
    """p(F) for a batch F [n, 3, 3] with per-item mu, lam [n]; model is one name or one per item.
    Triangles' F [n, 3, 2] go to the shell projections (``shell``)."""
    F = np.asarray(F, float)
    if F.shape[-1] == 2:
        from . import shell
        return shell.prox(model, F, mu, lam)
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,))
    lam = np.broadcast_to(np.asarray(lam, float), (n,))
    if not isinstance(model, str):
        P = np.zeros_like(F)
        for m, idx in by_model(model, n):
            P[idx] = prox(m, F[idx], mu[idx], lam[idx])
        return P
    if model == NEO_HOOKEAN:
        return _nh.prox(F, mu, lam)
    if model not in MODELS:
        raise ValueError(f"unknown model {model!r}")
    R, S, _, _ = polar_batch(F)
    if model == ARAP:
        return R
    c = corot_c(mu, lam)[:, None, None]
    return R @ (0.5 * (S + np.eye(3)) - c * (np.trace(S, axis1=1, axis2=2)[:, None, None] - 3.0) * np.eye(3))


def prox_derivatives(model, F, P, mu, lam):
    """dP/dF [n,9,9] (vec basis), dP/dmu [n,3,3], dP/dlam [n,3,3] at P = prox(model, F) (triangles:
    [n,6,6], [n,3,2], [n,3,2] from ``shell``)."""
    F = np.asarray(F, float)
    if F.shape[-1] == 2:
        from . import shell
        return shell.prox_derivatives(model, F, P, mu, lam)
    n = F.shape[0]
    mu = np.broadcast_to(np.asarray(mu, float), (n,))
    lam = np.broadcast_to(np.asarray(lam, float), (n,))
    if not isinstance(model, str):
        Jp, dmu, dlam = np.zeros((n, 9, 9)), np.zeros((n, 3, 3)), np.zeros((n, 3, 3))
        for m, idx in by_model(model, n):
            Jp[idx], dmu[idx], dlam[idx] = prox_derivatives(m, F[idx], None if P is None else P[idx], mu[idx],
                                                            lam[idx])
        return Jp, dmu, dlam
    if model == NEO_HOOKEAN:
        return _nh.prox_derivatives(F, P, mu, lam)
    Jp = np.zeros((n, 9, 9))
    dmu = np.zeros((n, 3, 3))
    dlam = np.zeros((n, 3, 3))
    I3 = np.eye(3)
    R, S, Q, s = polar_batch(F)
    c = corot_c(mu, lam)[:, None, None] if model == COROTATIONAL else None
    trS = np.trace(S, axis1=1, axis2=2)[:, None, None]
    K = 0.5 * (S + I3) - c * (trS - 3.0) * I3 if model == COROTATIONAL else None
    for m in range(9):
        e = np.zeros(9)
        e[m] = 1.0
        dR, dS = polar_differential_batch(R, S, Q, s, np.broadcast_to(unvec(e), F.shape))
        if model == ARAP:
            dP = dR
        else:
            dP = dR @ K + R @ (0.5 * dS - c * np.trace(dS, axis1=1, axis2=2)[:, None, None] * I3)
        Jp[:, :, m] = vec(dP)
    if model == COROTATIONAL:
        den = ((4.0 * mu + 3.0 * lam) ** 2)[:, None, None]
        dmu = R * ((trS - 3.0) * 2.0 * lam[:, None, None] / den)
        dlam = -R * ((trS - 3.0) * 2.0 * mu[:, None, None] / den)
    return Jp, dmu, dlam
