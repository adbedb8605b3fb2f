"""Smoothed Fischer-Burmeister contact: residuals, local solve and its Jacobians.

Test infrastructure (oracle); see the package docstring.

Per contact c (vertex v, frame rows n, t1, t2; all vectors below in frame coordinates):
    delta_n = n.q_v - d_n,   delta_f = [t1; t2](q_v - qbar_v) - d_f           (Eq. contact)
    phi_n = FB_eps(delta_n, lambda_n)
    phi_f = FB_eps(||delta_f||, mu lambda_n - gamma)
    lambda_f = -gamma t,  t = delta_f / ||delta_f||
with FB_eps(x, y) = x + y - sqrt(x^2 + y^2 + 2 eps^2)                          (Sec. 4.2).

Reading of the direction equation (Eq. constraint_direction): its linearisation along t is
identically zero, so lambda_f is parametrised by the signed multiplier gamma along -t.  The
paper's ||lambda_f|| equals gamma wherever its system has a solution (gamma >= 0); a contact
whose slip is too small for that (||delta_f|| < eps^2 / (mu lambda_n)) keeps the smooth
continuation gamma < 0.  A contact with mu = 0 is frictionless: it has no friction equation,
gamma = 0, and no dependence on mu (k_mu = 0).

Jacobians by implicit differentiation with the exact FB partials a = 1 - x/r, b = 1 - y/r,
r = sqrt(x^2 + y^2 + 2 eps^2) (App. A.2):
    K_c = -d lambda_c / d delta_c  (3x3),   k_mu = -d lambda_c / d mu  (3)    (Eq. final_diff_contact)
"""
from __future__ import annotations

import numpy as np


def fb(x, y, eps):
    return x + y - np.sqrt(x * x + y * y + 2.0 * eps * eps)


def fb_partials(x, y, eps):
    """(1 - x/r, 1 - y/r), written as (y^2 + 2 eps^2)/(r (r + x)) and (x^2 + 2 eps^2)/(r (r + y))
    so that neither loses digits when one argument dominates (the active-contact case)."""
    e2 = 2.0 * eps * eps
    r = np.sqrt(x * x + y * y + e2)
    return (y * y + e2) / (r * (r + x)), (x * x + e2) / (r * (r + y))


def tangent_dir(delta_f):
    nf = np.linalg.norm(delta_f)
    if nf == 0.0:
        return np.array([1.0, 0.0]), 0.0
    return delta_f / nf, nf


def local_solve(delta, mu, eps):
    """(lambda_n, gamma) solving phi_n = phi_f = 0 for a given frame-coordinate delta.

    FB_eps(x, y) = 0 iff x y = eps^2 with x + y > 0, so with delta_n > 0:
    lambda_n = eps^2 / delta_n and gamma = mu lambda_n - eps^2 / ||delta_f||.
    """
    dn = delta[0]
    if dn <= 0:
        raise ValueError("no local solution for delta_n <= 0")
    lam_n = eps * eps / dn
    if mu == 0.0:
        return lam_n, 0.0
    _, nf = tangent_dir(delta[1:])
    return lam_n, mu * lam_n - eps * eps / nf


def contact_force(lam_n, gamma, delta_f):
    """lambda_c (frame coordinates) from the multipliers."""
    t, _ = tangent_dir(delta_f)
    return np.array([lam_n, -gamma * t[0], -gamma * t[1]])


def contact_jacobians(delta, lam_n, gamma, mu, eps):
    """K_c = -d lambda_c/d delta (3x3) and k_mu = -d lambda_c/d mu (3), frame coordinates.

    Implicit differentiation of (phi_n, phi_f) = 0 for (lambda_n, gamma) as functions of
    (delta, mu), then lambda_c = (lambda_n, -gamma t(delta_f)).
    """
    dn = delta[0]
    an, bn = fb_partials(dn, lam_n, eps)
    # d phi_n = an d delta_n + bn d lambda_n = 0
    dlamn_ddelta = np.array([-an / bn, 0.0, 0.0])
    if mu == 0.0:
        K = np.zeros((3, 3))
        K[0, :] = -dlamn_ddelta
        return K, np.zeros(3)
    t, nf = tangent_dir(delta[1:])
    af, bf = fb_partials(nf, mu * lam_n - gamma, eps)
    # d phi_f = af d||delta_f|| + bf (mu d lambda_n + lambda_n d mu - d gamma) = 0
    dnorm_ddelta = np.array([0.0, t[0], t[1]])
    dgam_ddelta = mu * dlamn_ddelta + (af / bf) * dnorm_ddelta
    dgam_dmu = lam_n
    # d t / d delta_f = (I - t t^T) / ||delta_f||
    dt_ddf = (np.eye(2) - np.outer(t, t)) / nf
    dlam = np.zeros((3, 3))
    dlam[0] = dlamn_ddelta
    dlam[1:] = -np.outer(t, dgam_ddelta)
    dlam[1:, 1:] += -gamma * dt_ddf
    dlam_dmu = np.array([0.0, -dgam_dmu * t[0], -dgam_dmu * t[1]])
    return -dlam, -dlam_dmu


def paper_K_hat(delta, lam_n, gamma, mu):
    """The paper's on-manifold form R^T Khat R (Eq. final_diff_contact), R built from delta_f
    (App. A.1), for comparison with contact_jacobians at converged states."""
    t, nf = tangent_dir(delta[1:])
    R = np.array([[1.0, 0.0, 0.0], [0.0, t[0], t[1]], [0.0, -t[1], t[0]]])
    dn = delta[0]
    Kh = np.array([[lam_n / dn, 0.0, 0.0],
                   [-mu * lam_n / dn, (mu * lam_n - gamma) / nf, 0.0],
                   [0.0, 0.0, gamma / nf]])
    kmu = R.T @ np.array([0.0, lam_n, 0.0])
    if mu == 0.0:  # frictionless: no friction rows, no dependence on mu
        Kh[1:, :] = 0.0
        kmu = np.zeros(3)
    return R.T @ Kh @ R, kmu
