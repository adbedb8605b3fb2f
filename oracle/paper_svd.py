"""The paper's SVD closed form of the projection Jacobian, in FP64.

Test infrastructure (oracle); see the package docstring.  The adjoint in this oracle uses
the plain implicit-function form in ``prox``; this module exists so that the readings of
the closed form (Sec. 4.3 and App. B.0-B.4) are pinned against it on the CPU:

    dvecP/dvecF = (V (x) U) [D W D^T + Diag(vec M) + Diag(vec N) T] (V^T (x) U^T)

* Reading of a misprint: Sec. 4.3 and App. B.0 print the last term as Diag(vec M) T; the
  element-wise relation of App. B.0 has N_ij multiplying X_ji, so the term uses N.
* M_ij = (A_ij + B_ij)/2, N_ij = (A_ij - B_ij)/2 with A_ij = (theta_i-theta_j)/(sigma_i-sigma_j)
  and B_ij = (theta_i+theta_j)/(sigma_i+sigma_j) (App. B.0).  When |sigma_i - sigma_j| <= tau
  the divided difference A_ij is replaced by its limit, the symmetrised
  (W_ii + W_jj - W_ij - W_ji)/2 (App. B.4 gives W_ii - W_ij at exact degeneracy).
* Signed SVD: det U = det V = +1, the sign (if any) on sigma_3.
* theta solves g(theta) = mu(3 theta - 2 sigma - 1/theta) + lambda log(J) / theta = 0 (App. B.2/B.3),
  W = 2 mu (dg/dtheta)^{-1}, dtheta/dmu = -(dg/dtheta)^{-1}(3 theta - 2 sigma - 1/theta),
  dtheta/dlambda = -(dg/dtheta)^{-1} (log J / theta).
* The co-rotational and ARAP models (App. B.2) change only theta, W and the parameter
  derivatives (``model_theta``).  For ARAP, App. B.2 states M_ij = N_ij = 1/(sigma_i + sigma_j);
  App. B.0's definitions give M_ij = 1/(sigma_i + sigma_j) but N_ij = -1/(sigma_i + sigma_j)
  (A_ij = 0, B_ij = 2/(sigma_i + sigma_j)).  The definitions are taken; the polar-derivative
  oracle of ``models`` decides between the two.
"""
from __future__ import annotations

import numpy as np

# D x = vec(Diag x), T vec(X) = vec(X^T)  (App. B.1, 3D)
D_MAT = np.zeros((9, 3))
D_MAT[0, 0] = D_MAT[4, 1] = D_MAT[8, 2] = 1.0
T_MAT = np.zeros((9, 9))
for _r in range(3):
    for _k in range(3):
        T_MAT[_r + 3 * _k, _k + 3 * _r] = 1.0


def signed_svd(F):
    """F = U diag(s) V^T with det U = det V = +1 (sign of det F carried by s[2])."""
    U, s, Vt = np.linalg.svd(F)
    V = Vt.T.copy()
    U = U.copy()
    s = s.copy()
    if np.linalg.det(U) < 0:
        U[:, 2] *= -1
        s[2] *= -1
    if np.linalg.det(V) < 0:
        V[:, 2] *= -1
        s[2] *= -1
    return U, s, V


def nh_theta(sigma, mu, lam, tol=1e-15, max_iter=100):
    """Newton on g(theta) = 0 from theta = sigma, keeping theta > 0."""
    if np.any(sigma <= 0):
        raise ValueError("inverted element")
    th = sigma.astype(float).copy()
    for _ in range(max_iter):
        lJ = np.log(np.prod(th))
        g = mu * (3 * th - 2 * sigma - 1 / th) + lam * lJ / th
        if np.max(np.abs(g)) <= tol * mu:
            break
        Hd = np.diag(3 * mu + (mu - lam * lJ) / th ** 2) + lam * np.outer(1 / th, 1 / th)
        d = -np.linalg.solve(Hd, g)
        t = 1.0
        while np.any(th + t * d <= 0):
            t *= 0.5
        th = th + t * d
    return th


def nh_theta_derivatives(sigma, theta, mu, lam):
    """W = dtheta/dsigma, dtheta/dmu, dtheta/dlambda (App. B.2, B.3)."""
    lJ = np.log(np.prod(theta))
    a = 1.0 / theta
    H = np.diag(3 * mu + (mu - lam * lJ) * a ** 2) + lam * np.outer(a, a)
    Hinv = np.linalg.inv(H)
    W = 2.0 * mu * Hinv
    dmu = -Hinv @ (3 * theta - 2 * sigma - a)
    dlam = -Hinv @ (lJ * a)
    return W, dmu, dlam


def divided_difference_closed_form(theta, mu, lam, i, j):
    """A_ij for Neo-Hookean from the stationarity condition, without cancellation:
    subtracting the conditions for components i and j gives
    sigma_i - sigma_j = (theta_i - theta_j) [3 mu + (mu - lambda log J)/(theta_i theta_j)] / (2 mu)."""
    lJ = np.log(np.prod(theta))
    return 2.0 * mu / (3.0 * mu + (mu - lam * lJ) / (theta[i] * theta[j]))


def model_theta(model, sigma, mu, lam):
    """(theta, W, dtheta/dmu, dtheta/dlambda) of App. B.2/B.3 for 'neo_hookean', 'corotational'
    (g = 4 mu (theta - 1) + lambda tr(theta - 1) 1 - 2 mu (sigma - 1), H = dg/dtheta =
    4 mu I + lambda 1 1^T, dg/dmu = 2 (2 theta - sigma - 1), dg/dlambda = tr(theta - 1) 1) or
    'arap' (theta = 1, W = 0, no parameter dependence)."""
    sigma = np.asarray(sigma, float)
    if model == "neo_hookean":
        th = nh_theta(sigma, mu, lam)
        return (th,) + nh_theta_derivatives(sigma, th, mu, lam)
    if model == "corotational":
        one = np.ones(3)
        H = 4.0 * mu * np.eye(3) + lam * np.outer(one, one)
        th = one + np.linalg.solve(H, 2.0 * mu * (sigma - one))
        Hinv = np.linalg.inv(H)
        return (th, 2.0 * mu * Hinv, -Hinv @ (2.0 * (2.0 * th - sigma - one)),
                -Hinv @ (np.sum(th - one) * one))
    if model == "arap":
        return np.ones(3), np.zeros((3, 3)), np.zeros(3), np.zeros(3)
    raise ValueError(model)


def jacobian_svd(F, mu, lam, tau_sigma=1e-6, model="neo_hookean"):
    """9x9 dvecP/dvecF by the paper's SVD closed form (single F)."""
    U, s, V = signed_svd(F)
    th, W, _, _ = model_theta(model, s, mu, lam)
    M = np.zeros((3, 3))
    N = np.zeros((3, 3))
    tau = tau_sigma * max(1.0, np.max(np.abs(s)))
    for i in range(3):
        for j in range(3):
            if i == j:
                continue
            if abs(s[i] - s[j]) > tau:
                A = (th[i] - th[j]) / (s[i] - s[j])
            else:
                A = 0.5 * (W[i, i] + W[j, j] - W[i, j] - W[j, i])
            B = (th[i] + th[j]) / (s[i] + s[j])
            M[i, j] = 0.5 * (A + B)
            N[i, j] = 0.5 * (A - B)
    vecM = M.T.reshape(9)
    vecN = N.T.reshape(9)
    inner = D_MAT @ W @ D_MAT.T + np.diag(vecM) + np.diag(vecN) @ T_MAT
    K = np.kron(V, U)
    return K @ inner @ K.T


def prox_svd(F, mu, lam, model="neo_hookean"):
    """p(F) = U diag(theta) V^T (single F)."""
    U, s, V = signed_svd(F)
    th = model_theta(model, s, mu, lam)[0]
    return U @ np.diag(th) @ V.T
