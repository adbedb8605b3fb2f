"""Randomised properties of the oracle's local pieces (CPU only; hypothesis, where installed).

Each property holds for every input, so it complements the seeded pins with many random cases:
  - every model's projection Jacobian dp/dF is symmetric: p = F - grad Psi*(F) / w with Psi* the
    prox's Moreau envelope, so dp/dF = I - Hess Psi* / w;
  - the Neo-Hookean prox is isotropic and satisfies its stationarity condition;
  - the local contact solve zeroes both Fischer-Burmeister residuals, and its K_c matches a
    finite difference of lambda_c(delta).
"""
import numpy as np
import pytest

hyp = pytest.importorskip("hypothesis")
from hypothesis import given, settings  # noqa: E402
from hypothesis import strategies as st  # noqa: E402
from scipy.spatial.transform import Rotation  # noqa: E402

from oracle import contact as C  # noqa: E402
from oracle import models as Mo  # noqa: E402
from oracle.prox import grad_zeta  # noqa: E402

MU, LAM = 1e5 / (2 * 1.4), 1e5 * 0.4 / (1.4 * 0.2)


def _F(seed, strain):
    rng = np.random.default_rng(seed)
    R = Rotation.random(random_state=seed).as_matrix()
    F = R @ (np.eye(3) + strain * rng.standard_normal((3, 3)) / 3)
    return F if np.linalg.det(F) > 0.05 else R


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 2 ** 31 - 1), strain=st.floats(0.0, 0.6),
       model=st.sampled_from(["neo_hookean", "corotational", "arap"]))
def test_projection_jacobian_is_symmetric(seed, strain, model):
    F = _F(seed, strain)[None]
    P = Mo.prox(model, F, MU, LAM)
    Jp, _, _ = Mo.prox_derivatives(model, F, P, MU, LAM)
    assert np.abs(Jp[0] - Jp[0].T).max() <= 1e-9 * max(1.0, np.abs(Jp[0]).max())


@settings(max_examples=25, deadline=None)
@given(seed=st.integers(0, 2 ** 31 - 1), strain=st.floats(0.0, 0.6))
def test_neo_hookean_prox_is_stationary_and_isotropic(seed, strain):
    F = _F(seed, strain)
    P = Mo.prox("neo_hookean", F[None], MU, LAM)[0]
    g = 2 * MU * (P - F) + grad_zeta(P[None], MU, LAM)[0]
    assert np.abs(g).max() <= 1e-8 * MU
    Q = Rotation.random(random_state=seed + 1).as_matrix()
    assert np.allclose(Mo.prox("neo_hookean", (Q @ F)[None], MU, LAM)[0], Q @ P, atol=1e-11)
    assert np.allclose(Mo.prox("neo_hookean", (F @ Q)[None], MU, LAM)[0], P @ Q, atol=1e-11)


@settings(max_examples=40, deadline=None)
@given(dn=st.floats(1e-9, 1e-3), slip=st.floats(1e-9, 1e-3), ang=st.floats(0, 2 * np.pi),
       mu=st.sampled_from([0.0, 0.1, 0.5, 1.0]))
def test_local_contact_solve_and_its_jacobian(dn, slip, ang, mu):
    eps = 1e-4
    delta = np.array([dn, slip * np.cos(ang), slip * np.sin(ang)])
    lam_n, gam = C.local_solve(delta, mu, eps)
    assert abs(C.fb(delta[0], lam_n, eps)) <= 1e-12 * max(1.0, lam_n)
    if mu > 0:
        assert abs(C.fb(slip, mu * lam_n - gam, eps)) <= 1e-12 * max(1.0, mu * lam_n)
    K, _ = C.contact_jacobians(delta, lam_n, gam, mu, eps)

    def lam_c(d):
        ln, g = C.local_solve(d, mu, eps)
        return C.contact_force(ln, g, d[1:])

    h = 1e-6 * np.array([dn, slip, slip])
    fd = np.zeros((3, 3))
    for k in range(3):
        e = np.zeros(3)
        e[k] = h[k]
        fd[:, k] = -(lam_c(delta + e) - lam_c(delta - e)) / (2 * h[k])
    scale = np.abs(K).max()
    assert np.abs(fd - K).max() <= 1e-5 * scale
