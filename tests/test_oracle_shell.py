"""Pins of the oracle's triangle (shell) elements, App. B.1's 2D formulation, and of the isometric
bending term (Bergou et al. 2006):

* rest geometry: F of the rest shape (and of any rigid motion of it) has orthonormal columns; the
  areas and the lumped mass add up to the sheet's;
* the Neo-Hookean energy of a 3 x 2 P equals the volumetric energy of [P | n] (n the unit normal),
  its gradient and Hessian are the finite differences of the energy, and the prox is stationary,
  isotropic and the identity at rest;
* ARAP is the library's thin-SVD polar factor; co-rotational with lambda = 0 averages F and R, and
  otherwise minimises its 2D objective;
* dp/dF, dp/dmu, dp/dlambda match central differences, and dp/dF equals the thin-SVD closed form
  (per singular value theta(sigma), the in-plane 2 x 2 rule and the out-of-plane rows
  Y_3j = (theta_j / sigma_j) X_3j) built from theta alone;
* bending: for an isometric hinge of dihedral angle phi, ||K x|| = |e| 2 sin(phi/2); Q is symmetric
  positive semidefinite, vanishes on affine maps of a flat sheet and is invariant to rigid motions,
  and a sheet rolled into a cylinder of radius R stores energy proportional to 1/R^2;
* a whole cloth step: the adjoint matrix is the Jacobian of the reduced residual, and the adjoint
  gradients in E, nu, k_b, q_prev match central differences through the forward solve.
"""
import numpy as np
import pytest

import synth
from oracle import models as Mo
from oracle import prox as Pv
from oracle import shell as Sh
from tests._cases import make_step, rel

MU, LAM = 3.0e4, 7.0e4
MODELS = (Sh.NEO_HOOKEAN, Sh.COROTATIONAL, Sh.ARAP)


def _rot3(rng):
    q, r = np.linalg.qr(rng.standard_normal((3, 3)))
    q = q * np.sign(np.diag(r))
    return q if np.linalg.det(q) > 0 else -q


def _rot2(a):
    return np.array([[np.cos(a), -np.sin(a)], [np.sin(a), np.cos(a)]])


def _random_F(n, seed, strain=0.3):
    """3 x 2 deformation gradients U diag(sigma) V^T with sigma in [1 - strain, 1 + strain]."""
    rng = np.random.default_rng(seed)
    out = []
    for _ in range(n):
        U = _rot3(rng)[:, :2]
        V = _rot2(rng.uniform(0, 2 * np.pi))
        s = rng.uniform(1 - strain, 1 + strain, 2)
        out.append(U @ np.diag(s) @ V.T)
    return np.array(out)


# ---- rest geometry -----------------------------------------------------------------------------

def test_rest_deformation_gradient_is_orthonormal_and_masses_add_up():
    X, tris = synth.tri_grid(5, 4, 0.5, 0.4)
    rng = np.random.default_rng(0)
    inner = (X[:, 0] > 1e-9) & (X[:, 0] < 0.5 - 1e-9) & (X[:, 1] > 1e-9) & (X[:, 1] < 0.4 - 1e-9)
    X = X + rng.normal(0, 0.01, X.shape) * np.array([1, 1, 0]) * inner[:, None]  # irregular, flat, same outline
    m = Sh.TriMesh(X, tris, 2e-3)
    for q in (X, X @ _rot3(rng).T + rng.normal(size=3)):
        F = m.F(q)
        assert np.allclose(np.swapaxes(F, 1, 2) @ F, np.eye(2), atol=1e-12)
    assert abs(m.area.sum() - 0.5 * 0.4) < 1e-12 and np.all(m.area > 0)
    assert abs(m.lumped_mass(800.0).sum() - 800.0 * 2e-3 * 0.2) < 1e-12
    # G maps positions to vec6(F) with F's columns the edge vectors in the rest frame: an affine map
    # x -> A x sends F to A F_rest
    A = np.eye(3) + rng.normal(0, 0.1, (3, 3))
    assert np.allclose(m.F(X @ A.T), A @ m.F(X), atol=1e-12)


# ---- Neo-Hookean -------------------------------------------------------------------------------

def test_membrane_energy_is_the_volumetric_energy_of_the_extended_gradient():
    F = _random_F(6, 1, strain=0.4)
    for P in F:
        n = np.cross(P[:, 0], P[:, 1])
        n /= np.linalg.norm(n)
        assert abs(Sh.nh_zeta(P, MU, LAM) - Pv.zeta(np.column_stack([P, n]), MU, LAM)) < 1e-9 * MU


def test_gradient_and_hessian_are_finite_differences_of_the_energy():
    F = _random_F(4, 2, strain=0.4)
    eta = 1e-6
    for P in F:
        g = Sh.vec6(Sh.nh_grad(P, MU, LAM))
        H = Sh.nh_hess(P[None], np.array([MU]), np.array([LAM]))[0]
        gfd = np.array([(Sh.nh_zeta(P + eta * Sh.unvec6(e), MU, LAM) - Sh.nh_zeta(P - eta * Sh.unvec6(e), MU, LAM))
                        / (2 * eta) for e in np.eye(6)])
        Hfd = np.array([(Sh.vec6(Sh.nh_grad(P + eta * Sh.unvec6(e), MU, LAM))
                         - Sh.vec6(Sh.nh_grad(P - eta * Sh.unvec6(e), MU, LAM))) / (2 * eta) for e in np.eye(6)]).T
        assert np.max(np.abs(g - gfd)) < 1e-6 * MU
        assert np.max(np.abs(H - Hfd)) < 1e-5 * MU
        assert np.allclose(H, H.T, atol=1e-8 * MU)


@pytest.mark.parametrize("model", MODELS)
def test_prox_is_the_identity_at_rest_and_isotropic(model):
    rng = np.random.default_rng(3)
    Frest = np.array([_rot3(rng)[:, :2] for _ in range(3)])
    assert np.allclose(Sh.prox(model, Frest, MU, LAM), Frest, atol=1e-12)
    F = _random_F(5, 4, strain=0.4)
    P = Sh.prox(model, F, MU, LAM)
    R, V = _rot3(rng), _rot2(0.7)
    assert np.allclose(Sh.prox(model, R @ F @ V, MU, LAM), R @ P @ V, atol=1e-11)


def test_neo_hookean_prox_is_stationary():
    F = _random_F(6, 5, strain=0.5)
    P = Sh.nh_prox(F, MU, LAM)
    g = 2 * MU * (P - F) + Sh.nh_grad(P, MU, LAM)
    assert np.max(np.abs(g)) < 1e-9 * MU


# ---- ARAP and co-rotational ----------------------------------------------------------------------

def test_arap_is_the_thin_svd_polar_factor():
    F = _random_F(6, 6, strain=0.5)
    P = Sh.prox(Sh.ARAP, F, MU, LAM)
    for f, p in zip(F, P):
        U, _, Vt = np.linalg.svd(f, full_matrices=False)
        assert np.allclose(p, U @ Vt, atol=1e-12)


def test_corotational_with_zero_lambda_averages_F_and_its_rotation():
    F = _random_F(4, 7, strain=0.5)
    P = Sh.prox(Sh.COROTATIONAL, F, MU, 0.0)
    R = Sh.prox(Sh.ARAP, F, MU, 0.0)
    assert np.allclose(P, 0.5 * (F + R), atol=1e-12)


def test_corotational_prox_minimises_its_2d_objective():
    """mu ||P - F||^2 + mu ||S_P - I||^2 + lambda/2 (tr S_P - 2)^2, S_P the symmetric polar factor."""
    F = _random_F(4, 8, strain=0.4)
    P = Sh.prox(Sh.COROTATIONAL, F, MU, LAM)
    rng = np.random.default_rng(9)

    def obj(Pm, f):
        s = np.linalg.svd(Pm, compute_uv=False)
        return MU * np.sum((Pm - f) ** 2) + MU * np.sum((s - 1) ** 2) + 0.5 * LAM * (s.sum() - 2) ** 2

    for f, p in zip(F, P):
        f0 = obj(p, f)
        for _ in range(20):
            d = rng.standard_normal((3, 2)) * 1e-4
            assert obj(p + d, f) > f0 and obj(p - d, f) > f0


# ---- derivatives ---------------------------------------------------------------------------------

@pytest.mark.parametrize("model", MODELS)
def test_prox_derivatives_match_central_differences(model):
    F = _random_F(3, 10, strain=0.4)
    mu, lam = np.full(3, MU), np.full(3, LAM)
    P = Sh.prox(model, F, mu, lam)
    Jp, dmu, dlam = Sh.prox_derivatives(model, F, P, mu, lam)
    eta = 1e-6
    for m, e in enumerate(np.eye(6)):
        d = np.broadcast_to(Sh.unvec6(e), F.shape)
        fd = (Sh.prox(model, F + eta * d, mu, lam) - Sh.prox(model, F - eta * d, mu, lam)) / (2 * eta)
        assert np.max(np.abs(Jp[:, :, m] - Sh.vec6(fd))) < 1e-7
    fd_mu = (Sh.prox(model, F, mu * (1 + eta), lam) - Sh.prox(model, F, mu * (1 - eta), lam)) / (2 * eta * MU)
    fd_lam = (Sh.prox(model, F, mu, lam * (1 + eta)) - Sh.prox(model, F, mu, lam * (1 - eta))) / (2 * eta * LAM)
    assert np.max(np.abs(dmu - fd_mu)) < 1e-6 / MU
    assert np.max(np.abs(dlam - fd_lam)) < 1e-6 / LAM


def _theta(model, s):
    """The singular values of p(diag-form F): per model, theta(sigma) of the 2D stationarity."""
    if model == Sh.ARAP:
        return np.ones(2)
    if model == Sh.COROTATIONAL:
        return 0.5 * (s + 1) - LAM / (2 * (4 * MU + 2 * LAM)) * (s.sum() - 2)
    t = s.copy()  # Neo-Hookean: 2 mu (t - s) + mu (t - 1/t) + lam log(t1 t2) / t = 0, by Newton
    for _ in range(60):
        g = 2 * MU * (t - s) + MU * (t - 1 / t) + LAM * np.log(t.prod()) / t
        H = np.diag(3 * MU + MU / t ** 2 - LAM * np.log(t.prod()) / t ** 2) + LAM * np.outer(1 / t, 1 / t)
        t = t - np.linalg.solve(H, g)
    return t


@pytest.mark.parametrize("model", MODELS)
def test_jacobian_equals_the_thin_svd_closed_form(model):
    """F = U diag(sigma) V^T (U 3 x 2, completed by the normal u_3): in the basis X = [U u_3]^T dF V,
    dP maps the diagonal by d theta / d sigma, the off-diagonal pair by (theta_1 -/+ theta_2) /
    (sigma_1 -/+ sigma_2) on its symmetric/skew parts, and the out-of-plane row by theta_j / sigma_j."""
    F = _random_F(3, 11, strain=0.4)
    mu, lam = np.full(3, MU), np.full(3, LAM)
    Jp, _, _ = Sh.prox_derivatives(model, F, Sh.prox(model, F, mu, lam), mu, lam)
    eta = 1e-6
    for f, J in zip(F, Jp):
        U, s, Vt = np.linalg.svd(f, full_matrices=False)
        Uf = np.column_stack([U, np.cross(U[:, 0], U[:, 1])])
        th = _theta(model, s)
        dth = np.array([(_theta(model, s + eta * e) - _theta(model, s - eta * e)) / (2 * eta) for e in np.eye(2)]).T
        Jc = np.zeros((6, 6))
        for m, e in enumerate(np.eye(6)):
            X = Uf.T @ Sh.unvec6(e) @ Vt.T           # 3 x 2
            Y = np.zeros((3, 2))
            Y[0, 0], Y[1, 1] = dth @ np.array([X[0, 0], X[1, 1]])
            sym, skw = 0.5 * (X[0, 1] + X[1, 0]), 0.5 * (X[0, 1] - X[1, 0])
            a = (th[0] - th[1]) / (s[0] - s[1])
            b = (th[0] + th[1]) / (s[0] + s[1])
            Y[0, 1], Y[1, 0] = a * sym + b * skw, a * sym - b * skw
            Y[2, :] = th / s * X[2, :]
            Jc[:, m] = Sh.vec6(Uf @ Y @ Vt)
        assert np.max(np.abs(J - Jc)) < 1e-7, np.max(np.abs(J - Jc))


def test_degenerate_triangles_are_rejected():
    F = np.array([[[1.0, 2.0], [0.0, 0.0], [0.0, 0.0]]])
    for model in MODELS:
        with pytest.raises(Sh.DegenerateElement):
            Sh.prox(model, F, MU, LAM)


def test_triangle_gradients_dispatch_from_the_volumetric_entry_points():
    F = _random_F(3, 12)
    for model in MODELS:
        assert np.array_equal(Mo.prox(model, F, MU, LAM), Sh.prox(model, F, MU, LAM))


# ---- isometric bending -------------------------------------------------------------------------

@pytest.mark.parametrize("shift", [0.0, 0.4])
@pytest.mark.parametrize("phi", [0.3, 1.0, 2.0])
def test_hinge_stencil_measures_the_dihedral_angle(phi, shift):
    """Two rest-flat triangles sharing an edge of length L, one folded by phi about it (an
    isometry): ||sum_a K_a x_a|| = L 2 sin(phi/2), whatever the triangles' shapes."""
    L = 1.3
    X = np.array([[0, 0, 0], [L, 0, 0], [0.5, 0.8, 0], [0.4 + shift, -0.7, 0]], float)
    m = Sh.TriMesh(X, np.array([[0, 1, 2], [1, 0, 3]]), 1e-3)
    (idx, K, A), = m.bending_stencils()
    assert abs(A - 0.5 * L * (0.8 + 0.7)) < 1e-12
    c, s = np.cos(phi), np.sin(phi)
    x = X.copy()
    x[3] = np.array([[1, 0, 0], [0, c, -s], [0, s, c]]) @ X[3]
    assert abs(np.linalg.norm(K @ x[list(idx)]) - L * 2 * np.sin(phi / 2)) < 1e-12


def test_bending_matrix_structure():
    nx, ny = 5, 4
    X, tris = synth.tri_grid(nx, ny, 0.5, 0.4)
    rng = np.random.default_rng(1)
    X = X + rng.normal(0, 0.01, X.shape) * np.array([1, 1, 0])
    m = Sh.TriMesh(X, tris, 1e-3)
    n_edges = nx * (ny + 1) + ny * (nx + 1) + nx * ny
    assert len(m.bending_stencils()) == n_edges - 2 * (nx + ny)  # one stencil per interior edge
    Q = m.bending_matrix().toarray()
    assert np.allclose(Q, Q.T, atol=0)
    assert np.linalg.eigvalsh(Q).min() > -1e-9 * np.abs(Q).max()
    # zero on every affine image of the flat rest sheet
    for _ in range(3):
        A, b = rng.normal(size=(3, 3)), rng.normal(size=3)
        y = (X @ A.T + b).reshape(-1)
        assert np.linalg.norm(Q @ y) < 1e-10 * np.abs(Q).max() * np.linalg.norm(y)
    # invariant to rigid motions of a bent configuration
    x = X + np.column_stack([0 * X[:, 0], 0 * X[:, 0], np.sin(6 * X[:, 0]) * 0.05])
    R, b = _rot3(rng), rng.normal(size=3)
    e0 = x.reshape(-1) @ Q @ x.reshape(-1)
    e1 = (x @ R.T + b).reshape(-1) @ Q @ (x @ R.T + b).reshape(-1)
    assert e0 > 0 and abs(e1 - e0) < 1e-10 * e0


def test_rolled_sheet_energy_scales_as_inverse_radius_squared():
    """A sheet rolled isometrically onto a cylinder of radius R: every fold angle is proportional to
    1/R, so x^T Q x = sum 3/A_e ||K_e x||^2 goes as 4 sin^2(c / 2R) ~ 1/R^2."""
    X, tris = synth.tri_grid(12, 6, 0.6, 0.3)
    Q = Sh.TriMesh(X, tris, 1e-3).bending_matrix()

    def energy(Rc):
        t = X[:, 0] / Rc
        x = np.column_stack([Rc * np.sin(t), X[:, 1], Rc * (1 - np.cos(t))])
        return x.reshape(-1) @ (Q @ x.reshape(-1))
    e1, e2, e4 = energy(1.0), energy(2.0), energy(4.0)
    assert abs(e1 / e2 - 4.0) < 0.02 and abs(e2 / e4 - 4.0) < 0.005


# ---- a whole cloth step ------------------------------------------------------------------------

CLOTH = dict(n=5, size=0.1, radius=0.04, height=0.002, mu=0.3, bend=2e-4, E=3e4)


def _cloth_case(k):
    from tests._cases import step_case
    return step_case("cloth_drape", k, **CLOTH)


def test_cloth_adjoint_matrix_is_the_jacobian_of_the_reduced_residual():
    pb, st, s, q_prev, v_prev = _cloth_case(3)
    assert st.nc > 0 and st.Qb is not None
    qt = st.qtilde(q_prev, v_prev, np.zeros_like(q_prev))
    A = st.adjoint_matrix(s, q_prev)[0].toarray()

    def Rq(q):
        ln, g = st.local_multipliers(q, q_prev)
        return st.residual(q, ln, g, q_prev, qt)[:st.N] * st.h ** 2
    q0 = s.q.ravel()
    Jfd = np.zeros((st.N, st.N))
    for j in range(st.N):
        e = np.zeros(st.N)
        e[j] = 1e-11  # below the contact gaps, above the residual's rounding
        Jfd[:, j] = (Rq((q0 + e).reshape(-1, 3)) - Rq((q0 - e).reshape(-1, 3))) / 2e-11
    assert np.max(np.abs(Jfd - A)) < 1e-6 * np.max(np.abs(A))


def test_cloth_step_gradient_matches_central_differences():
    """L = ||q - q_target||^2 through the oracle's forward cloth step (contact set and frames
    frozen) against the adjoint's dL/dE, dL/dnu, dL/dk_b, dL/dmu and dL/dq_prev."""
    pb, st, base, q_prev, v_prev = _cloth_case(3)
    sc = pb.scene
    qt = pb.q_target
    g = st.adjoint(base, q_prev, 2 * (base.q - qt), np.zeros_like(qt))

    def L(E=sc.E, nu=sc.nu, bend=sc.bend, mu=None, dq=0.0):
        s2 = make_step(sc, st.ct, E=E, nu=nu, bend=bend)
        r = s2.forward(q_prev + dq, v_prev, mu_c=None if mu is None else np.full(st.nc, mu), q_init=base.q)
        assert r.residual < 1e-8
        return np.sum((r.q - qt) ** 2)

    def cd(f, eta):
        return (f(eta) - f(-eta)) / (2 * eta)

    E0, nu0, kb = sc.E[0], sc.nu[0], sc.bend
    assert rel(g["dL_dE"].sum(), cd(lambda e: L(E=E0 + e), 1e-6 * E0)) < 1e-6
    # a membrane's loss hardly depends on nu: a smaller step drowns in the forward's residual
    assert rel(g["dL_dnu"].sum(), cd(lambda e: L(nu=nu0 + e), 1e-4 * nu0)) < 1e-6
    assert rel(g["dL_dbend"], cd(lambda e: L(bend=kb + e), 1e-6 * kb)) < 1e-6
    mu0 = st.ct.mu[0]
    assert rel(g["dL_dmu_contact"].sum(), cd(lambda e: L(mu=mu0 + e), 1e-4 * mu0)) < 1e-4
    d = np.random.default_rng(15).normal(size=qt.shape)
    d /= np.linalg.norm(d)
    assert rel(np.sum(g["dL_dq_prev"] * d), cd(lambda e: L(dq=e * d), 1e-9)) < 1e-4
