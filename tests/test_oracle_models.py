"""Pins of the co-rotational and ARAP oracle (App. B.2/B.3) on the CPU.

The oracle builds both projections from the polar decomposition; each test checks it against
something else: the prox's definition as a minimiser, the nearest-rotation property, a closed
form by a matrix square root, the paper's printed W and parameter derivatives, finite
differences, and the SVD closed form of App. B.0.
"""
import numpy as np
import pytest
from scipy.linalg import sqrtm
from scipy.spatial.transform import Rotation

from oracle import models as Mo
from oracle import paper_svd as S
from oracle.model import unvec, vec
from tests._cases import rel, step_case, make_step

MU, LAM = 1e5 / (2 * 1.4), 1e5 * 0.4 / (1.4 * 0.2)  # E = 1e5, nu = 0.4
MODELS = (Mo.COROTATIONAL, Mo.ARAP)


def _random_F(seed, n, strain=0.3):
    rng = np.random.default_rng(seed)
    R = Rotation.random(n, random_state=seed).as_matrix()
    return np.einsum("nij,njk->nik", R, np.eye(3) + strain * rng.standard_normal((n, 3, 3)) / 3)


def _rotation_by_sqrtm(F):
    """The polar rotation F (F^T F)^{-1/2}, by a matrix square root."""
    return F @ np.linalg.inv(np.real(sqrtm(F.T @ F)))


def test_batched_polar_and_its_differential_match_the_library_routines():
    """The step's batched polar factors (eigendecomposition of F^T F) and their differential (the
    Sylvester equation solved in the eigenbasis of S) against scipy's polar and solve_sylvester."""
    F = _random_F(16, 5, strain=0.5)
    R, Sb, Q, s = Mo.polar_batch(F)
    dF = np.random.default_rng(17).standard_normal(F.shape)
    dR, dS = Mo.polar_differential_batch(R, Sb, Q, s, dF)
    for i in range(len(F)):
        R1, S1 = Mo.polar_one(F[i])
        assert np.allclose(R[i], R1, atol=1e-13) and np.allclose(Sb[i], S1, atol=1e-13)
        dR1, dS1 = Mo.polar_differential(R1, S1, dF[i])
        assert np.allclose(dR[i], dR1, atol=1e-12) and np.allclose(dS[i], dS1, atol=1e-12)
        assert np.allclose(dS[i], dS[i].T, atol=1e-12) and np.allclose(R1.T @ dR[i], -(R1.T @ dR[i]).T, atol=1e-12)


def test_corotational_with_zero_lambda_averages_F_and_its_rotation():
    """lambda = 0: theta = (sigma + 1)/2, so p(F) = (F + R)/2."""
    F = _random_F(1, 6)
    P = Mo.prox(Mo.COROTATIONAL, F, MU, 0.0)
    for f, p in zip(F, P):
        assert np.allclose(p, 0.5 * (f + _rotation_by_sqrtm(f)), atol=1e-12)


def test_arap_is_the_nearest_rotation():
    F = _random_F(2, 5)
    P = Mo.prox(Mo.ARAP, F, MU, LAM)
    Q = Rotation.random(400, random_state=3).as_matrix()
    for f, p in zip(F, P):
        assert np.allclose(p.T @ p, np.eye(3), atol=1e-13) and abs(np.linalg.det(p) - 1) < 1e-13
        assert np.allclose(p, _rotation_by_sqrtm(f), atol=1e-11)
        d0 = np.sum((f - p) ** 2)
        assert np.all(np.sum((Q - f) ** 2, axis=(1, 2)) >= d0 - 1e-12)


def test_corotational_prox_minimises_its_objective():
    """p(F) minimises mu ||P - F||^2 + zeta(P) with zeta from P's singular values (App. B.2):
    the finite-difference gradient vanishes and every nearby P costs more."""
    F = _random_F(4, 4, strain=0.5)
    P = Mo.prox(Mo.COROTATIONAL, F, MU, LAM)
    rng = np.random.default_rng(5)

    def obj(Pm, f):
        return MU * np.sum((Pm - f) ** 2) + Mo.zeta_corotational(Pm, MU, LAM)

    for f, p in zip(F, P):
        f0 = obj(p, f)
        eta = 1e-6
        grad = np.array([(obj(p + eta * unvec(e), f) - obj(p - eta * unvec(e), f)) / (2 * eta) for e in np.eye(9)])
        assert np.max(np.abs(grad)) < 1e-6 * MU
        for _ in range(20):
            d = unvec(rng.standard_normal(9)) * 1e-3
            assert obj(p + d, f) > f0 and obj(p - d, f) > f0


def test_corotational_theta_W_and_parameter_derivatives_match_the_printed_forms():
    """On F = diag(sigma): theta by finite differences gives W = I/2 - lambda/(2(4mu+3lambda)) 11^T
    (App. B.2), and d theta/d mu, d theta/d lambda equal -H^{-1} dg/dmu, -H^{-1} dg/dlambda (App. B.3)."""
    sig = np.array([1.3, 0.85, 0.7])

    def theta(s, mu=MU, lam=LAM):
        return np.diag(Mo.prox(Mo.COROTATIONAL, np.diag(s)[None], mu, lam)[0])

    eta = 1e-6
    W = np.stack([(theta(sig + eta * e) - theta(sig - eta * e)) / (2 * eta) for e in np.eye(3)], axis=1)
    W_print = 0.5 * np.eye(3) - LAM / (2 * (4 * MU + 3 * LAM)) * np.ones((3, 3))
    assert np.allclose(W, W_print, atol=1e-8)
    th, Wm, dmu, dlam = S.model_theta(Mo.COROTATIONAL, sig, MU, LAM)
    assert np.allclose(th, theta(sig), atol=1e-14) and np.allclose(Wm, W_print, atol=1e-14)
    fd_mu = (theta(sig, mu=MU * (1 + eta)) - theta(sig, mu=MU * (1 - eta))) / (2 * eta * MU)
    fd_lam = (theta(sig, lam=LAM * (1 + eta)) - theta(sig, lam=LAM * (1 - eta))) / (2 * eta * LAM)
    assert rel(dmu, fd_mu) < 1e-7 and rel(dlam, fd_lam) < 1e-7
    # the oracle's own parameter derivatives: on a positive diagonal F, R = I and dP/dmu = diag(dtheta/dmu)
    _, dPm, dPl = Mo.prox_derivatives(Mo.COROTATIONAL, np.diag(sig)[None], None, MU, LAM)
    assert np.allclose(dPm[0], np.diag(dmu), atol=1e-14 * np.abs(dmu).max() + 1e-20)
    assert np.allclose(dPl[0], np.diag(dlam), atol=1e-14 * np.abs(dlam).max() + 1e-20)


@pytest.mark.parametrize("model", MODELS)
def test_jacobians_match_finite_differences(model):
    F = _random_F(7, 3, strain=0.4)
    P = Mo.prox(model, F, MU, LAM)
    Jp, dmu, dlam = Mo.prox_derivatives(model, F, P, MU, LAM)
    eta = 1e-6
    for i in range(len(F)):
        Jfd = np.zeros((9, 9))
        for m in range(9):
            e = eta * unvec(np.eye(9)[m])
            Jfd[:, m] = (vec(Mo.prox(model, (F[i] + e)[None], MU, LAM)[0])
                         - vec(Mo.prox(model, (F[i] - e)[None], MU, LAM)[0])) / (2 * eta)
        assert np.allclose(Jp[i], Jfd, atol=1e-8)
        d = (Mo.prox(model, F[i:i + 1], MU * (1 + eta), LAM)[0] - Mo.prox(model, F[i:i + 1], MU * (1 - eta), LAM)[0])
        assert np.allclose(dmu[i], d / (2 * eta * MU), atol=1e-14)
        d = (Mo.prox(model, F[i:i + 1], MU, LAM * (1 + eta))[0] - Mo.prox(model, F[i:i + 1], MU, LAM * (1 - eta))[0])
        assert np.allclose(dlam[i], d / (2 * eta * LAM), atol=1e-14)


@pytest.mark.parametrize("model", MODELS)
@pytest.mark.parametrize("seed,strain", [(8, 0.05), (9, 0.4)])
def test_svd_closed_form_with_the_model_theta_equals_the_polar_derivative(model, seed, strain):
    """App. B.0's (V (x) U)[D W D^T + Diag(vec M) + Diag(vec N) T](V (x) U)^T with the model's theta
    and W equals the oracle's polar-decomposition Jacobian.  For ARAP this fixes the sign of N."""
    F = _random_F(seed, 3, strain)
    P = Mo.prox(model, F, MU, LAM)
    Jp, _, _ = Mo.prox_derivatives(model, F, P, MU, LAM)
    for i in range(len(F)):
        assert np.allclose(S.jacobian_svd(F[i], MU, LAM, model=model), Jp[i], atol=1e-11)
        assert np.allclose(S.prox_svd(F[i], MU, LAM, model=model), P[i], atol=1e-12)


def test_arap_with_the_printed_N_sign_is_wrong():
    """M_ij = N_ij = 1/(sigma_i + sigma_j) as printed in App. B.2 does not give the ARAP Jacobian."""
    F = _random_F(10, 1)[0]
    U, s, V = S.signed_svd(F)
    M = np.array([[0 if i == j else 1 / (s[i] + s[j]) for j in range(3)] for i in range(3)])
    inner = np.diag(M.T.reshape(9)) + np.diag(M.T.reshape(9)) @ S.T_MAT
    K = np.kron(V, U)
    J_printed = K @ inner @ K.T
    Jp, _, _ = Mo.prox_derivatives(Mo.ARAP, F[None], None, MU, LAM)
    assert np.max(np.abs(J_printed - Jp[0])) > 0.1


@pytest.mark.parametrize("model", MODELS)
def test_arap_and_corotational_rotation_invariance(model):
    """p(Q F) = Q p(F) and p(F Q) = p(F) Q for rotations Q (isotropy)."""
    F = _random_F(11, 2)
    Q = Rotation.random(1, random_state=12).as_matrix()[0]
    P = Mo.prox(model, F, MU, LAM)
    assert np.allclose(Mo.prox(model, Q @ F, MU, LAM), Q @ P, atol=1e-12)
    assert np.allclose(Mo.prox(model, F @ Q, MU, LAM), P @ Q, atol=1e-12)


def test_inverted_elements_are_rejected():
    F = np.diag([1.0, 1.0, -0.5])[None]
    for model in MODELS:
        with pytest.raises(Mo.InvertedElement):
            Mo.prox(model, F, MU, LAM)


@pytest.mark.parametrize("model", MODELS)
def test_whole_step_gradient_matches_central_differences(model):
    """Central differences of L = ||q - q_target||^2 through the oracle forward step under the
    model, with the contact set and frames frozen, against the oracle adjoint."""
    pb, st, base, q_prev, v_prev = step_case("cube_drop", 2, model)
    sc = pb.scene
    qt = pb.q_target
    g = st.adjoint(base, q_prev, 2 * (base.q - qt), np.zeros_like(qt))

    def L(E=sc.E, nu=sc.nu, mu=None, dq=0.0):
        s2 = make_step(sc, st.ct, E=E, nu=nu, model=model)
        r = s2.forward(q_prev + dq, v_prev, mu_c=None if mu is None else np.full(st.nc, mu), q_init=base.q)
        assert r.residual < 1e-8
        return np.sum((r.q - qt) ** 2)

    def cd(f, eta):
        return (f(eta) - f(-eta)) / (2 * eta)

    E0, nu0 = sc.E[0], sc.nu[0]
    assert rel(g["dL_dE"].sum(), cd(lambda e: L(E=E0 + e), 1e-6 * E0)) < 1e-6
    assert rel(g["dL_dnu"].sum(), cd(lambda e: L(nu=nu0 + e), 1e-6 * nu0)) < 1e-6
    mu0 = st.ct.mu[0]
    # the forward stops at a residual near 1e-10, so a smaller step drowns in solver noise
    assert rel(g["dL_dmu_contact"].sum(), cd(lambda e: L(mu=mu0 + e), 1e-4 * mu0)) < 1e-4
    d = np.random.default_rng(14).normal(size=qt.shape)
    d /= np.linalg.norm(d)
    assert rel(np.sum(g["dL_dq_prev"] * d), cd(lambda e: L(dq=e * d), 1e-9)) < 1e-4


def test_per_tet_models_dispatch_by_group():
    """A per-item model array gives each item its own model's projection and derivatives."""
    F = _random_F(15, 6)
    names = np.array([Mo.NEO_HOOKEAN, Mo.COROTATIONAL, Mo.ARAP] * 2)
    P = Mo.prox(names, F, MU, LAM)
    Jp, dmu, dlam = Mo.prox_derivatives(names, F, P, MU, LAM)
    for i, m in enumerate(names):
        Pi = Mo.prox(str(m), F[i:i + 1], MU, LAM)
        Ji, mi, li = Mo.prox_derivatives(str(m), F[i:i + 1], Pi, MU, LAM)
        assert np.array_equal(P[i], Pi[0]) and np.array_equal(Jp[i], Ji[0])
        assert np.array_equal(dmu[i], mi[0]) and np.array_equal(dlam[i], li[0])
    with pytest.raises(ValueError):
        Mo.prox(np.array(["stvk"] * 6), F, MU, LAM)


def test_arap_gradients_in_E_and_nu_are_tied_through_mu():
    """ARAP ignores lambda, so per tet dL/dnu = -E / (1 + nu) dL/dE (both act through mu alone)."""
    pb, st, s, q_prev, v_prev = step_case("cube_drop", 2, Mo.ARAP)
    g = st.adjoint(s, q_prev, 2 * (s.q - pb.q_target), np.zeros_like(pb.q_target))
    expect = -g["dL_dE"] * st.E / (1.0 + st.nu)
    assert np.allclose(g["dL_dnu"], expect, rtol=1e-12, atol=1e-14 * np.abs(expect).max())
    assert np.abs(g["dL_dlamL"]).max() == 0.0
