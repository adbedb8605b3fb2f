"""Pins of the FP64 oracle against what the paper and the mathematics fix (CPU only).

Each test checks an oracle function against something other than itself: values printed in
the paper (tests/golden), closed forms, finite differences, brute force, invariants.
"""
import os

import numpy as np
import pytest

import synth
from oracle import contact as C
from oracle import paper_svd as S
from oracle.model import unvec, vec
from oracle.prox import grad_zeta, prox, prox_derivatives
from oracle.woodbury import contact_jacobian_matrix, woodbury_apply
from tests._cases import make_step, rel, step_case

GOLD = os.path.join(os.path.dirname(__file__), "golden")
MU, LAM = 1e5 / (2 * 1.4), 1e5 * 0.4 / (1.4 * 0.2)  # E = 1e5, nu = 0.4


def _read_golden(name):
    out, key = {}, None
    for line in open(os.path.join(GOLD, name)):
        line = line.strip()
        if not line or line.startswith("#"):
            continue
        parts = line.split()
        if len(parts) == 1:
            key = parts[0]
            out[key] = []
        elif key is None or (len(parts) == 2 and not parts[0].lstrip("-").replace(".", "").isdigit()):
            out[parts[0]] = float(parts[1])
        else:
            out[key].append([float(p) for p in parts])
    return out


# ---- conventions ------------------------------------------------------------------------

def test_vec_conventions_match_printed_D_T():
    """App. B.1 prints D and T; they fix vec = column stacking."""
    g = _read_golden("app_b1_D_T.txt")
    D = np.array(g["D"])
    T = np.array(g["T"])
    assert np.array_equal(D, S.D_MAT) and np.array_equal(T, S.T_MAT)
    rng = np.random.default_rng(0)
    x = rng.normal(size=3)
    X = rng.normal(size=(3, 3))
    assert np.allclose(D @ x, vec(np.diag(x)))
    assert np.allclose(T @ vec(X), vec(X.T))
    assert np.allclose(D.T @ vec(X), np.diag(X))


# ---- Neo-Hookean prox -------------------------------------------------------------------

def test_prox_rest_is_identity():
    P = prox(np.eye(3)[None], MU, LAM)
    assert np.allclose(P[0], np.eye(3), atol=1e-15)


def test_prox_stationarity_and_isotropy():
    F = synth.random_deformation_gradients(50, seed=1, strain=0.1)
    P = prox(F, MU, LAM)
    g = 2 * MU * (P - F) + grad_zeta(P, MU, LAM)
    assert np.max(np.abs(g)) <= 1e-12 * MU
    # isotropy: P shares F's singular vectors (U^T P V is diagonal)
    for f, p in zip(F, P):
        U, s, V = S.signed_svd(f)
        M = U.T @ p @ V
        assert np.max(np.abs(M - np.diag(np.diag(M)))) < 1e-12


def test_prox_matches_svd_route():
    """Plain 9-D minimisation == U diag(theta(sigma)) V^T with the App. B.2 scalar equation."""
    F = synth.random_deformation_gradients(20, seed=2, strain=0.2)
    P = prox(F, MU, LAM)
    for f, p in zip(F, P):
        assert np.allclose(S.prox_svd(f, MU, LAM), p, atol=1e-13)


def _J_rest_expected(mu, lam):
    """dp/dF at F = I: 1 on skew, 1/2 on symmetric traceless, 2mu/(4mu+3lam) on volume."""
    I9 = np.eye(9)
    T = S.T_MAT
    Psym = 0.5 * (I9 + T)
    Pskew = 0.5 * (I9 - T)
    vI = vec(np.eye(3))
    Pvol = np.outer(vI, vI) / 3.0
    return Pskew + 0.5 * (Psym - Pvol) + 2 * mu / (4 * mu + 3 * lam) * Pvol


def test_jacobian_at_rest_closed_form():
    F = np.eye(3)[None]
    P = prox(F, MU, LAM)
    Jp, _, _ = prox_derivatives(F, P, MU, LAM)
    assert np.allclose(Jp[0], _J_rest_expected(MU, LAM), atol=1e-13)


def test_jacobian_at_rotation_closed_form():
    R = synth.random_deformation_gradients(5, seed=3, strain=0.0)
    P = prox(R, MU, LAM)
    Jp, _, _ = prox_derivatives(R, P, MU, LAM)
    J0 = _J_rest_expected(MU, LAM)
    for r, j in zip(R, Jp):
        IR = np.kron(np.eye(3), r)
        assert np.allclose(j, IR @ J0 @ IR.T, atol=1e-12)


def test_jacobian_matches_finite_differences():
    F = synth.random_deformation_gradients(6, seed=4, strain=0.15)
    P = prox(F, MU, LAM)
    Jp, dmu, dlam = prox_derivatives(F, P, MU, LAM)
    eta = 1e-6
    for i in range(len(F)):
        Jfd = np.zeros((9, 9))
        for m in range(9):
            e = np.zeros(9)
            e[m] = eta
            Jfd[:, m] = (vec(prox((F[i] + unvec(e))[None], MU, LAM)[0])
                         - vec(prox((F[i] - unvec(e))[None], MU, LAM)[0])) / (2 * eta)
        assert np.max(np.abs(Jfd - Jp[i])) < 1e-8
        d = (prox(F[i:i + 1], MU * (1 + eta), LAM)[0] - prox(F[i:i + 1], MU * (1 - eta), LAM)[0]) / (2 * eta * MU)
        assert np.max(np.abs(d - dmu[i])) < 1e-6 * np.max(np.abs(d))
        d = (prox(F[i:i + 1], MU, LAM * (1 + eta))[0] - prox(F[i:i + 1], MU, LAM * (1 - eta))[0]) / (2 * eta * LAM)
        assert np.max(np.abs(d - dlam[i])) < 1e-6 * np.max(np.abs(d))


def test_jacobian_symmetric_and_positive():
    """dp/dF is symmetric (it is 2 mu H^{-1}); its spectrum lies in [0, 1] only where
    grad^2 zeta >= 0 (Sec. 4.4), which Neo-Hookean satisfies at rest but not under strain."""
    F = synth.random_deformation_gradients(20, seed=5, strain=0.05)
    P = prox(F, MU, LAM)
    Jp, _, _ = prox_derivatives(F, P, MU, LAM)
    for j in Jp:
        assert np.allclose(j, j.T, atol=1e-12)
        ev = np.linalg.eigvalsh(0.5 * (j + j.T))
        assert ev.min() > 0 and ev.max() < 1.2
    J0, _, _ = prox_derivatives(np.eye(3)[None], np.eye(3)[None], MU, LAM)
    ev = np.linalg.eigvalsh(J0[0])
    assert ev.min() > 0 and ev.max() <= 1 + 1e-12


# ---- the paper's SVD closed form (readings of Sec. 4.3 / App. B) -------------------------

@pytest.mark.parametrize("seed,strain", [(6, 0.05), (7, 0.3)])
def test_paper_svd_jacobian_equals_plain_definition(seed, strain):
    F = synth.random_deformation_gradients(10, seed=seed, strain=strain)
    P = prox(F, MU, LAM)
    Jp, _, _ = prox_derivatives(F, P, MU, LAM)
    for f, j in zip(F, Jp):
        assert np.max(np.abs(S.jacobian_svd(f, MU, LAM) - j)) < 1e-10


@pytest.mark.parametrize("delta", [1e-2, 1e-4, 1e-6, 1e-7, 1e-9, 0.0])
def test_paper_svd_jacobian_near_degenerate(delta):
    """App. B.4 limits: no blow-up across the tau switch, including exact degeneracy."""
    rng = np.random.default_rng(8)
    Q = synth.random_deformation_gradients(2, seed=9, strain=0.0)
    F = Q[0] @ np.diag([1.0, 1.0 + delta, 1.0 + 2 * delta]) @ Q[1].T * (1.0 + 0.01 * rng.random())
    P = prox(F[None], MU, LAM)
    Jp, _, _ = prox_derivatives(F[None], P, MU, LAM)
    assert np.max(np.abs(S.jacobian_svd(F, MU, LAM) - Jp[0])) < 1e-8


def test_printed_T_term_with_M_is_wrong():
    """Reading of the misprint: with Diag(vec M) T (as printed) the Jacobian differs from the
    plain definition; with Diag(vec N) T it agrees (previous test)."""
    F = synth.random_deformation_gradients(1, seed=10, strain=0.2)[0]
    U, s, V = S.signed_svd(F)
    th = S.nh_theta(s, MU, LAM)
    W, _, _ = S.nh_theta_derivatives(s, th, MU, LAM)
    M = np.zeros((3, 3))
    for i in range(3):
        for j in range(3):
            if i != j:
                M[i, j] = (s[i] * th[i] - s[j] * th[j]) / (s[i] ** 2 - s[j] ** 2)
    vM = vec(M)
    K = np.kron(V, U)
    J_printed = K @ (S.D_MAT @ W @ S.D_MAT.T + np.diag(vM) + np.diag(vM) @ S.T_MAT) @ K.T
    P = prox(F[None], MU, LAM)
    Jp, _, _ = prox_derivatives(F[None], P, MU, LAM)
    assert np.max(np.abs(J_printed - Jp[0])) > 1e-2


def test_divided_difference_closed_form():
    """(theta_i - theta_j)/(sigma_i - sigma_j) == 2mu / (3mu + (mu - lam log J)/(theta_i theta_j))."""
    for sig in ([1.3, 0.9, 0.7], [1.05, 1.0, 0.98], [2.0, 1.5, 0.5]):
        s = np.array(sig)
        th = S.nh_theta(s, MU, LAM)
        for i, j in ((0, 1), (0, 2), (1, 2)):
            dd = (th[i] - th[j]) / (s[i] - s[j])
            assert abs(dd - S.divided_difference_closed_form(th, MU, LAM, i, j)) < 1e-9 * abs(dd)


def test_corotational_W_rest_matches_paper_formula():
    """At F = I the NH W equals the co-rotational W = I/2 - lam/(2(4mu+3lam)) 11^T (App. B.2)."""
    s = np.ones(3)
    th = S.nh_theta(s, MU, LAM)
    W, _, _ = S.nh_theta_derivatives(s, th, MU, LAM)
    assert np.allclose(W, 0.5 * np.eye(3) - LAM / (2 * (4 * MU + 3 * LAM)) * np.ones((3, 3)), atol=1e-14)


# ---- contact ----------------------------------------------------------------------------

def _manifold_point(kind, mu=0.5, eps=1e-4):
    if kind == "stick":
        dn, nf, lam = 1e-8 / 0.4, 1e-7, 0.4
    elif kind == "slide":
        dn, nf, lam = 1e-8 / 0.3, 3e-4, 0.3
    else:  # separating within the margin, tiny slip (gamma < 0 continuation)
        dn, nf, lam = 1e-3, 2e-5, 1e-8 / 1e-3
    ang = 0.7
    delta = np.array([dn, nf * np.cos(ang), nf * np.sin(ang)])
    lam_n, gam = C.local_solve(delta, mu, eps)
    return delta, lam_n, gam


@pytest.mark.parametrize("kind", ["stick", "slide", "separate"])
def test_contact_K_matches_finite_differences(kind):
    mu, eps = 0.5, 1e-4
    delta, lam_n, gam = _manifold_point(kind, mu, eps)
    assert abs(C.fb(delta[0], lam_n, eps)) < 1e-12 * lam_n
    K, kmu = C.contact_jacobians(delta, lam_n, gam, mu, eps)

    def lam_of(d, m=mu):
        ln, g = C.local_solve(d, m, eps)
        return C.contact_force(ln, g, d[1:])
    Kfd = np.zeros((3, 3))
    for j in range(3):
        e = np.zeros(3)
        e[j] = 1e-6 * abs(delta[j]) + 1e-12
        Kfd[:, j] = -(lam_of(delta + e) - lam_of(delta - e)) / (2 * e[j])
    assert np.max(np.abs(Kfd - K)) < 1e-6 * np.max(np.abs(K))
    kfd = -(lam_of(delta, mu * (1 + 1e-6)) - lam_of(delta, mu * (1 - 1e-6))) / (2e-6 * mu)
    assert np.max(np.abs(kfd - kmu)) < 1e-6 * max(np.max(np.abs(kmu)), 1e-30)


@pytest.mark.parametrize("kind", ["stick", "slide"])
def test_contact_K_equals_paper_ratio_form_on_manifold(kind):
    """On the converged manifold the exact partials reduce to the paper's R^T Khat R (C-9)."""
    delta, lam_n, gam = _manifold_point(kind)
    K, kmu = C.contact_jacobians(delta, lam_n, gam, 0.5, 1e-4)
    Kp, kmup = C.paper_K_hat(delta, lam_n, gam, 0.5)
    assert np.allclose(K, Kp, rtol=1e-8, atol=1e-8 * np.max(np.abs(K)))
    assert np.allclose(kmu, kmup, rtol=1e-12)


def test_frictionless_contact_block():
    """mu = 0: K = diag(lambda_n / delta_n, 0, 0) in the contact frame (Sec. 4.4, frictionless)."""
    delta = np.array([2.5e-8, 1e-4, -3e-5])
    lam_n, gam = C.local_solve(delta, 0.0, 1e-4)
    K, kmu = C.contact_jacobians(delta, lam_n, gam, 0.0, 1e-4)
    assert np.allclose(K, np.diag([lam_n / delta[0], 0, 0]), rtol=1e-9)
    assert np.all(kmu == 0)


def test_eps_consistency_scaling():
    """App. A.2: at a forward-converged contact, a backward eps != forward eps scales the
    active-row K entry by eps_fwd^2/eps_bwd^2 and the inactive-row one by the reciprocal."""
    g = _read_golden("app_a2_eps_consistency.txt")
    e_f = np.sqrt(g["two_eps_fwd_sq"] / 2)
    e_b = np.sqrt(g["two_eps_bwd_sq"] / 2)
    # active: y = lambda_n = O(1), x = delta_n = eps_f^2 / y
    lam_n = 0.7
    d_act = np.array([e_f ** 2 / lam_n, 1.0, 0.0])
    Kf, _ = C.contact_jacobians(d_act, lam_n, 0.0, 0.0, e_f)
    Kb, _ = C.contact_jacobians(d_act, lam_n, 0.0, 0.0, e_b)
    assert abs(Kb[0, 0] / Kf[0, 0] / g["active_row_factor"] - 1) < 1e-3
    # inactive: x = delta_n = O(1), y = lambda_n = eps_f^2 / x
    dn = 0.7
    d_in = np.array([dn, 1.0, 0.0])
    Kf, _ = C.contact_jacobians(d_in, e_f ** 2 / dn, 0.0, 0.0, e_f)
    Kb, _ = C.contact_jacobians(d_in, e_f ** 2 / dn, 0.0, 0.0, e_b)
    assert abs(Kb[0, 0] / Kf[0, 0] / g["inactive_row_factor"] - 1) < 1e-3


# ---- Woodbury identity ------------------------------------------------------------------

def test_woodbury_equals_dense_inverse():
    pb, st, s, q_prev, _ = step_case("two_tet", 1)
    Amat, pc = st.adjoint_matrix(s, q_prev)
    A = pc["A_el"].toarray()
    # the preconditioner's elastic part is A (no Delta A); use it as in Eq. woodbury_formula
    mu_L, _ = st.lame()
    from oracle.model import elastic_matrix
    A = elastic_matrix(st.mesh, st.mass, mu_L, st.h).toarray()
    J = contact_jacobian_matrix(st.mesh.n_verts, st.ct.vertex, st.ct.frame)
    Kt = np.swapaxes(pc["K"], 1, 2)  # transposed system
    Kfull = np.zeros((J.shape[0],) * 2)
    for c in range(st.nc):
        Kfull[3 * c:3 * c + 3, 3 * c:3 * c + 3] = Kt[c]
    dense = np.linalg.inv(A + st.h ** 2 * J.T @ Kfull @ J)
    r = np.random.default_rng(11).normal(size=A.shape[0])
    assert rel(woodbury_apply(A, J, Kt, st.h, r), dense @ r) < 1e-12
    # no contacts -> A^{-1}
    assert rel(woodbury_apply(A, J, 0 * Kt, st.h, r), np.linalg.solve(A, r)) < 1e-14


# ---- the adjoint matrix and the whole-step gradient --------------------------------------

def test_adjoint_matrix_is_jacobian_of_reduced_residual():
    """script_A = d R_q / d q with the multipliers eliminated by the local contact solve."""
    pb, st, s, q_prev, v_prev = step_case("two_tet", 1)
    qt = st.qtilde(q_prev, v_prev, np.zeros_like(q_prev))
    Amat, _ = st.adjoint_matrix(s, q_prev)

    def Rq(q):
        ln, g = st.local_multipliers(q, q_prev)
        return st.residual(q, ln, g, q_prev, qt)[:st.N] * st.h ** 2
    q0 = s.q.ravel()
    Jfd = np.zeros((st.N, st.N))
    for j in range(st.N):
        e = np.zeros(st.N)
        e[j] = 1e-12  # the normal gaps are ~2e-8 m: the step must be far below them
        Jfd[:, j] = (Rq((q0 + e).reshape(-1, 3)) - Rq((q0 - e).reshape(-1, 3))) / 2e-12
    A = Amat.toarray()
    assert np.max(np.abs(Jfd - A)) < 1e-6 * np.max(np.abs(A))


def test_contact_free_adjoint_is_spd_and_above_mass():
    """Sec. 4.4: with no contact, script_A = A - Delta A is symmetric and >= M where
    grad^2 zeta >= 0 -- exactly so at rest.  Under strain Neo-Hookean is not convex and the
    near-rigid rotation modes may dip slightly below M; script_A itself stays SPD."""
    from oracle.step import State
    pb, st, s, q_prev, _ = step_case("cube_drop", 0)
    assert st.nc == 0
    M = np.diag(np.repeat(st.mass, 3))
    rest = State(pb.scene.X.copy(), np.zeros(0), np.zeros(0))
    A0 = st.adjoint_matrix(rest, pb.scene.X)[0].toarray()
    assert np.allclose(A0, A0.T, atol=1e-12 * np.abs(A0).max())
    ev0 = np.linalg.eigvalsh(A0 - M)
    assert ev0.min() > -1e-12 * ev0.max()
    A = st.adjoint_matrix(s, q_prev)[0].toarray()
    assert np.allclose(A, A.T, atol=1e-12 * np.abs(A).max())
    ev = np.linalg.eigvalsh(A - M)
    assert ev.min() > -1e-4 * ev.max()
    assert np.linalg.eigvalsh(A).min() > 0


def test_frictional_adjoint_is_nonsymmetric_and_transpose_matters():
    """Sec. 4.4: with friction script_A is not symmetric; solving with script_A instead of
    script_A^T changes the gradient (the adjoint needs the transpose)."""
    import scipy.sparse.linalg as spla
    pb, st, s, q_prev, _ = step_case("cube_drop", 2)
    A, _ = st.adjoint_matrix(s, q_prev)
    asym = abs(A - A.T).max() / abs(A).max()
    assert asym > 1e-6
    b = np.random.default_rng(12).normal(size=st.N)
    z = spla.spsolve(A.T.tocsc(), b)
    z_wrong = spla.spsolve(A.tocsc(), b)
    assert rel(z_wrong, z) > 1e-5


@pytest.mark.parametrize("k", [2, 5])
def test_whole_step_gradient_matches_central_differences(k):
    """Central differences (Sec. 5.1) of L = ||q - q_target||^2 through the oracle forward
    step, with the contact set and frames frozen, against the oracle adjoint."""
    pb, st, base, q_prev, v_prev = step_case("cube_drop", k)
    sc = pb.scene
    qt = pb.q_target
    g = st.adjoint(base, q_prev, 2 * (base.q - qt), np.zeros_like(qt))

    def L(E=sc.E, nu=sc.nu, mu=None, dq=0.0, dv=0.0, df=0.0):
        s2 = make_step(sc, st.ct, E=E, nu=nu)
        r = s2.forward(q_prev + dq, v_prev + dv, f_ctrl=np.zeros_like(qt) + df,
                       mu_c=None if mu is None else np.full(st.nc, mu), q_init=base.q)
        assert r.residual < 1e-8
        return np.sum((r.q - qt) ** 2)

    def cd(f, eta):
        return (f(eta) - f(-eta)) / (2 * eta)

    E0, nu0 = sc.E[0], sc.nu[0]
    assert rel(g["dL_dE"].sum(), cd(lambda e: L(E=E0 + e), 1e-6 * E0)) < 1e-6
    assert rel(g["dL_dnu"].sum(), cd(lambda e: L(nu=nu0 + e), 1e-6 * nu0)) < 1e-6
    mu0 = st.ct.mu[0]
    assert rel(g["dL_dmu_contact"].sum(), cd(lambda e: L(mu=mu0 + e), 1e-6 * mu0)) < 1e-4
    rng = np.random.default_rng(13)
    for key, arg, scale in (("dL_dq_prev", "dq", 1e-3), ("dL_dv_prev", "dv", 1e-2), ("dL_dfext", "df", 1e-2)):
        d = rng.normal(size=qt.shape)
        d /= np.linalg.norm(d)
        fd = cd(lambda e: L(**{arg: e * d}), 1e-6 * scale)
        assert rel(np.sum(g[key] * d), fd) < 1e-4, key


# ---- per-tet actuation (constant active stress a_i d_i d_i^T) ---------------------------------

def _face_normal_forces(X, tet, P):
    """Nodal forces of a constant first Piola stress on one tet from its faces: vertex a gets
    P (A_a n_a) / 3, with A_a n_a the outward area vector of the face opposite a."""
    out = np.zeros((4, 3))
    for a in range(4):
        b, c, d = [tet[k] for k in range(4) if k != a]
        av = 0.5 * np.cross(X[c] - X[b], X[d] - X[b])
        if av @ (X[tet[a]] - X[b]) > 0:
            av = -av
        out[a] = P @ av / 3.0
    return out


def test_stress_force_matches_face_area_vectors():
    from oracle.actuation import stress_force
    from oracle.model import Mesh
    rng = np.random.default_rng(21)
    X = rng.normal(size=(4, 3))
    tet = np.array([0, 1, 2, 3])
    if np.linalg.det(np.stack([X[1] - X[0], X[2] - X[0], X[3] - X[0]], axis=1)) < 0:
        tet = np.array([0, 2, 1, 3])
    P = rng.normal(size=(3, 3))  # not symmetric: a transposed operand shows
    f = stress_force(Mesh(X, tet[None]), P[None])
    ref = _face_normal_forces(X, tet, P)
    assert np.abs(f[tet] - ref).max() < 1e-12 * np.abs(ref).max()


def test_actuation_force_has_no_net_force_or_torque_at_rest():
    from oracle.actuation import actuation_force
    from oracle.model import Mesh
    X, tets = synth.hex_tet_mesh(3, 2, 2, 0.01)
    act, fibre = synth.random_actuation(len(tets), seed=3)
    f = actuation_force(Mesh(X, tets), act, fibre)
    scale = np.abs(f).max()
    assert scale > 0
    assert np.abs(f.sum(axis=0)).max() < 1e-12 * scale * len(X)
    assert np.abs(np.cross(X, f).sum(axis=0)).max() < 1e-12 * scale * len(X) * np.abs(X).max()


def test_actuation_gradient_matches_central_differences():
    """dL/da through the whole oracle step (contacts and frames frozen), directional check."""
    from oracle.actuation import actuation_force, actuation_gradient
    pb, st, base, q_prev, v_prev = step_case("cube_drop", 2)
    sc = pb.scene
    qt = pb.q_target
    act, fibre = synth.random_actuation(st.mesh.n_tets, seed=5)
    act = act.astype(float)

    def solve(a):
        r = st.forward(q_prev, v_prev, f_ctrl=actuation_force(st.mesh, a, fibre), q_init=base.q)
        assert r.residual < 1e-8
        return r

    s0 = solve(act)
    g = st.adjoint(s0, q_prev, 2 * (s0.q - qt), np.zeros_like(qt))
    ga = actuation_gradient(st.mesh, g["z"], fibre, sc.h)
    # the chain through f_ext: dL/da = (dL/df_ext) . df_act/da
    e = np.zeros(st.mesh.n_tets)
    e[7] = 1.0
    assert abs(ga[7] - np.sum(g["dL_dfext"] * actuation_force(st.mesh, e, fibre))) < 1e-12 * np.abs(ga).max()
    rng = np.random.default_rng(22)
    d = rng.normal(size=act.shape)
    d /= np.linalg.norm(d)
    eta = 1e-6 * np.abs(act).max()
    fd = (np.sum((solve(act + eta * d).q - qt) ** 2) - np.sum((solve(act - eta * d).q - qt) ** 2)) / (2 * eta)
    assert rel(ga @ d, fd) < 1e-5


# ---- eps -> 0 limit: the smoothed step tends to the equality-constrained (bilateral) step ----------

def test_resting_frictionless_contacts_converge_to_the_bilateral_kkt_gradient():
    """As eps -> 0 a resting frictionless contact enforces delta_n = 0: state, multipliers and
    adjoint solution z tend to those of the KKT system of the constrained step (dense LU), at
    the O(eps^2) rate of lambda_n = eps^2 / delta_n."""
    from oracle.bilateral import constrained_adjoint, constrained_step
    pb = synth.cube_drop(cells=2, drop=1e-4, v_sigma=0.0, mu=0.0)
    sc = pb.scene
    q_prev, v_prev = pb.q0.copy(), pb.v0.copy()
    ct = sc.contacts(q_prev)
    assert ct.n == 9
    seed = np.random.default_rng(3).normal(size=q_prev.shape)
    runs = []
    for eps in (1e-2, 1e-3, 1e-4, 1e-5):
        st = make_step(sc, ct, eps=eps)
        s = st.forward(q_prev, v_prev)
        assert s.residual < 1e-10 and np.all(s.lam_n > 0)
        runs.append((s, st.adjoint(s, q_prev, seed, np.zeros_like(seed))["z"]))
    q_star, lam_star = constrained_step(st, q_prev, v_prev, runs[-1][0].q)
    assert np.all(lam_star > 0)
    z_star = constrained_adjoint(st, q_star, q_prev, seed)
    ez = [rel(z, z_star) for _, z in runs]
    eq = [rel(s.q - q_prev, q_star - q_prev) for s, _ in runs]
    el = [rel(s.lam_n, lam_star) for s, _ in runs]
    for e in (ez, eq, el):
        assert all(e[i + 1] < e[i] / 30 for i in range(len(e) - 1)), e
    assert ez[-1] < 1e-6 and eq[-1] < 1e-6 and el[-1] < 1e-6


def test_separating_contacts_converge_to_the_contact_free_gradient():
    """Contacts that open during the step carry lambda_n = eps^2/delta_n -> 0 and a tangential
    stiffness ~ eps^2/||delta_f||^2 (both FB arguments are small): the adjoint solution tends to
    that of the same step without contacts, at the O(eps^2) rate."""
    from oracle.bilateral import _free
    pb = synth.cube_drop(cells=2, drop=1e-3, v_sigma=0.0, mu=0.3)
    sc = pb.scene
    q_prev = pb.q0.copy()
    v_prev = np.tile([0.3, 0.0, 0.5], (len(q_prev), 1))  # moving up and sideways: every gap opens
    ct = sc.contacts(q_prev)
    assert ct.n == 9
    seed = np.random.default_rng(4).normal(size=q_prev.shape)
    free = _free(make_step(sc, ct))
    s0 = free.forward(q_prev, v_prev)
    z0 = free.adjoint(s0, q_prev, seed, np.zeros_like(seed))["z"]
    errs = []
    for eps in (1e-2, 1e-3, 1e-4, 1e-5):
        st = make_step(sc, ct, eps=eps)
        s = st.forward(q_prev, v_prev)
        assert s.residual < 1e-10
        errs.append(rel(st.adjoint(s, q_prev, seed, np.zeros_like(seed))["z"], z0))
    assert all(errs[i + 1] < errs[i] / 30 for i in range(len(errs) - 1)) and errs[-1] < 1e-7, errs


# ---- continuity of dL/dmu through the slip threshold ----------------------------------------

def test_friction_gradient_is_continuous_through_the_stick_slip_threshold():
    """A block sliding down the 20 degree incline (5 cm/s) is stopped within the step once
    mu exceeds ~0.91.  Sweeping mu across that threshold, the adjoint dL/dmu must equal the
    central difference of L(mu) at every sample (sliding, transition and sticking alike), and
    its integral must reproduce the change of L: a jump or a wrong value in the transition fails
    one of the two."""
    pb = synth.beam_incline(nx=4, ny=2, nz=2)
    sc = pb.scene
    q_prev = pb.q0.copy()
    t1 = sc.planes[0].frame[1]                      # up the slope
    v_prev = np.tile(-0.05 * t1, (len(q_prev), 1))  # sliding down
    ct = sc.contacts(q_prev)
    st = make_step(sc, ct)
    com_t = q_prev.mean(axis=0) + np.array([0.001, 0.0, 0.0])

    def run(mu, grad=True):
        mu_c = np.full(ct.n, mu)
        s = st.forward(q_prev, v_prev, mu_c=mu_c)
        assert s.residual < 1e-10
        com = s.q.mean(axis=0)
        L = np.sum((com - com_t) ** 2)
        if not grad:
            return L
        seed = np.tile(2 * (com - com_t) / len(s.q), (len(s.q), 1))
        g = st.adjoint(s, q_prev, seed, np.zeros_like(seed), mu_c=mu_c)["dL_dmu_region"][0]
        slip = min(np.linalg.norm(st.delta(s.q, q_prev, c)[1:]) for c in range(ct.n))
        return L, g, slip

    mus = np.linspace(0.84, 0.98, 15)
    res = [run(m) for m in mus]
    Ls = np.array([r[0] for r in res])
    gs = np.array([r[1] for r in res])
    slips = np.array([r[2] for r in res])
    assert slips[0] > 10 * slips[-1]          # sliding at the start of the sweep, sticking at its end
    assert abs(gs[0]) > 5 * abs(gs[-1])       # and the friction gradient changes regime with it
    for m, g in zip(mus[::3], gs[::3]):
        eta = 1e-6
        fd = (run(m + eta, False) - run(m - eta, False)) / (2 * eta)
        assert abs(g - fd) <= 1e-5 * abs(g), (m, g, fd)
    # trapezoid integral of dL/dmu against L(mu_end) - L(mu_start)
    integral = np.sum(0.5 * (gs[1:] + gs[:-1]) * np.diff(mus))
    assert abs(integral - (Ls[-1] - Ls[0])) <= 5e-3 * abs(Ls[-1] - Ls[0])


# ---- frame completion: gradients do not depend on the choice of t1, t2 ---------------------

@pytest.mark.parametrize("k", [2, 5])
def test_gradients_are_invariant_to_the_tangent_frame(k):
    """Rotating each contact's (t1, t2) about its normal by its own angle leaves the converged
    state and every gradient unchanged: only the frame coordinates of lambda_f rotate."""
    import dataclasses
    pb, st, s, q_prev, v_prev = step_case("cube_drop", k)
    qt = pb.q_target
    ct = st.ct
    ang = np.random.default_rng(31).uniform(0, 2 * np.pi, ct.n)
    frame = ct.frame.copy()
    c_, s_ = np.cos(ang)[:, None], np.sin(ang)[:, None]
    frame[:, 1] = c_ * ct.frame[:, 1] + s_ * ct.frame[:, 2]
    frame[:, 2] = -s_ * ct.frame[:, 1] + c_ * ct.frame[:, 2]
    rot = make_step(pb.scene, dataclasses.replace(ct, frame=frame))
    s2 = rot.forward(q_prev, v_prev, q_init=s.q)
    assert s2.residual < 1e-8
    assert np.max(np.abs(s2.q - s.q)) <= 1e-12 * np.max(np.abs(s.q - q_prev))
    dq = 2 * (s.q - qt)
    dv = np.random.default_rng(32).normal(size=qt.shape) * 1e-3
    g1 = st.adjoint(s, q_prev, dq, dv)
    g2 = rot.adjoint(s2, q_prev, dq, dv)
    for key in ("z", "dL_dq_prev", "dL_dv_prev", "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu_contact"):
        assert rel(g2[key], g1[key]) < 1e-9, key


@pytest.mark.parametrize("k", [2, 5])
def test_paper_epsilon_variant(k):
    """The paper's own smoothing, 2 eps^2 = 1e-12 (config 1 otherwise unchanged): the forward stops
    at its rounding floor (residual ~1e-6 of h^2 |M g|, the contacts being ~1e4 times stiffer than at
    eps = 1e-4), and the adjoint still matches central differences in E."""
    from tests._cases import rollout
    eps = np.sqrt(0.5e-12)
    pb, q_prev, v_prev = rollout("cube_drop", k)
    sc = pb.scene
    ct = sc.contacts(q_prev)
    st = make_step(sc, ct, eps=eps)
    s = st.forward(q_prev, v_prev)
    assert s.residual < 1e-5
    qt = pb.q_target
    g = st.adjoint(s, q_prev, 2 * (s.q - qt), np.zeros_like(qt))

    def L(E):
        r = make_step(sc, ct, E=E, eps=eps).forward(q_prev, v_prev, q_init=s.q)
        return np.sum((r.q - qt) ** 2)

    E0, eta = sc.E[0], 1e-6
    fd = (L(E0 * (1 + eta)) - L(E0 * (1 - eta))) / (2 * eta * E0)
    assert rel(g["dL_dE"].sum(), fd) < 1e-7


@pytest.mark.parametrize("k", [2, 5])
def test_frictionless_adjoint_is_symmetric_positive_definite(k):
    """Sec. 4.4: without friction the contact blocks are R^T diag(lambda_n/delta_n, 0, 0) R, so
    script_A stays symmetric and (here) positive definite."""
    import dataclasses
    pb, st, s, q_prev, v_prev = step_case("cube_drop", k)
    ct0 = dataclasses.replace(st.ct, mu=np.zeros(st.nc))
    st0 = make_step(pb.scene, ct0)
    s0 = st0.forward(q_prev, v_prev)
    assert s0.residual < 1e-8 and st0.nc > 0
    A, _ = st0.adjoint_matrix(s0, q_prev)
    assert abs(A - A.T).max() <= 1e-13 * abs(A).max()
    np.linalg.cholesky(A.toarray())  # raises if not positive definite
