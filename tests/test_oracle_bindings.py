"""Pins of the bilateral binding oracle (Eq. binding, single-vertex attachments) on the CPU:
whole-step central differences of every gradient, and the stiff limit E_b -> 0 against the
hard attachment solved as an equality-constrained KKT system (dense LU)."""
import numpy as np
import pytest

from oracle.binding import Bindings
from oracle.bilateral import constrained_adjoint, constrained_step, vertex_rows
from oracle.step import Step
from tests._cases import rel, rollout

H_TOP = 4  # bound vertices: the top corners of the cube


def _top_corners(X):
    z = X[:, 2]
    top = np.nonzero(z >= z.max() - 1e-12)[0]
    xy = X[top, :2]
    corners = [top[np.argmin(s * xy[:, 0] + t * xy[:, 1])] for s in (1, -1) for t in (1, -1)]
    return np.array(corners)


def _case(k, compliance, shift=1e-3, lateral=2e-4, model="neo_hookean"):
    """Cube-drop step k with its four top corners attached to targets lifted by ``shift`` and
    moved sideways by ~``lateral`` (larger sideways pulls turn the sliding contacts, which the
    forward's line search refuses)."""
    pb, q_prev, v_prev = rollout("cube_drop", k)
    sc = pb.scene
    verts = _top_corners(sc.X)
    target = (q_prev[verts] + np.array([0.0, 0.0, shift])
              + lateral * np.random.default_rng(3).standard_normal((4, 3)))
    bd = Bindings(verts, np.full(4, compliance), target)
    ct = sc.contacts(q_prev)
    st = Step(sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h, sc.gravity, ct, sc.eps, model, bd)
    return pb, st, bd, q_prev, v_prev


def test_binding_multiplier_and_blocks_follow_the_compliant_spring():
    """lambda_b = -(q_v - d_b)/E_b; the adjoint matrix grows by h^2/E_b I_3 on bound vertices."""
    pb, st, bd, q_prev, v_prev = _case(0, 1e-4)
    q = q_prev + 1e-3
    lam = bd.multipliers(q)
    assert np.allclose(lam, -(q[bd.vertex] - bd.target) / 1e-4)
    Kb = bd.matrix_term(st.h, st.mesh.n_verts).toarray()
    for v in range(st.mesh.n_verts):
        blk = Kb[3 * v:3 * v + 3, 3 * v:3 * v + 3]
        expect = st.h ** 2 / 1e-4 * np.eye(3) if v in bd.vertex else np.zeros((3, 3))
        assert np.allclose(blk, expect)
    assert np.count_nonzero(Kb) == 3 * H_TOP


@pytest.mark.parametrize("k", [0, 2])
def test_whole_step_gradients_match_central_differences(k):
    """Central differences of L = ||q - q_target||^2 through the oracle forward step with the
    bindings, against the adjoint: d_b (a random direction), each E_b, q_prev (a random direction)."""
    pb, st, bd, q_prev, v_prev = _case(k, 1e-4)
    qt = pb.q_target
    base = st.forward(q_prev, v_prev)
    assert base.residual < 1e-9
    g = st.adjoint(base, q_prev, 2 * (base.q - qt), np.zeros_like(qt))

    def L(target=bd.target, compliance=bd.compliance, dq=0.0):
        b2 = Bindings(bd.vertex, compliance, target)
        s2 = Step(st.mesh.X, st.mesh.tets, st.E, st.nu, st.density, st.h, st.gravity, st.ct, st.eps, st.model, b2)
        r = s2.forward(q_prev + dq, v_prev, q_init=base.q)
        assert r.residual < 1e-9
        return np.sum((r.q - qt) ** 2)

    def cd(f, eta):
        return (f(eta) - f(-eta)) / (2 * eta)

    d = np.random.default_rng(11).standard_normal(bd.target.shape)
    d /= np.linalg.norm(d)
    assert rel(np.sum(g["dL_dbinding_target"] * d), cd(lambda e: L(target=bd.target + e * d), 1e-7)) < 1e-5
    for b in range(bd.n):
        e_b = np.zeros(bd.n)
        e_b[b] = 1.0
        fd = cd(lambda e: L(compliance=bd.compliance + e * e_b), 1e-4 * bd.compliance[b])
        assert rel(g["dL_dcompliance"][b], fd) < 1e-5, b
    dq = np.random.default_rng(12).standard_normal(qt.shape)
    dq /= np.linalg.norm(dq)
    assert rel(np.sum(g["dL_dq_prev"] * dq), cd(lambda e: L(dq=e * dq), 1e-8)) < 1e-5


def test_stiff_bindings_converge_to_the_hard_attachment():
    """E_b -> 0: the state tends to the step with q_v = d_b held exactly (KKT, dense LU), and
    dL/dd_b = h^2 z_v / E_b tends to the KKT multiplier of the adjoint, both at rate O(E_b)."""
    errs_q, errs_g = [], []
    hard = None
    for E in (1e-4, 1e-5, 1e-6, 1e-7):
        pb, st, bd, q_prev, v_prev = _case(0, E)
        assert st.nc == 0
        qt = pb.q_target
        s = st.forward(q_prev, v_prev, tol=1e-12)
        g = st.adjoint(s, q_prev, 2 * (s.q - qt), np.zeros_like(qt))
        if hard is None:
            Nm = vertex_rows(st.mesh.n_verts, bd.vertex)
            q_h, _ = constrained_step(st, q_prev, v_prev, s.q, Nm=Nm, d=bd.target)
            assert np.allclose(q_h[bd.vertex], bd.target, atol=1e-14)
            _, w_l = constrained_adjoint(st, q_h, q_prev, 2 * (q_h - qt), Nm=Nm, with_multiplier=True)
            hard = (q_h, w_l.reshape(-1, 3))
        errs_q.append(rel(s.q - q_prev, hard[0] - q_prev))
        errs_g.append(rel(g["dL_dbinding_target"], hard[1]))
    for e in (errs_q, errs_g):
        assert all(e[i + 1] < e[i] / 8 for i in range(len(e) - 1)), e
    assert errs_q[-1] < 1e-4 and errs_g[-1] < 1e-4, (errs_q, errs_g)


def test_soft_bindings_vanish():
    """E_b -> infinity: the bound step's gradients tend to the free step's."""
    pb, st, bd, q_prev, v_prev = _case(2, 1e6)
    free = Step(st.mesh.X, st.mesh.tets, st.E, st.nu, st.density, st.h, st.gravity, st.ct, st.eps)
    qt = pb.q_target
    s1 = st.forward(q_prev, v_prev)
    s0 = free.forward(q_prev, v_prev)
    g1 = st.adjoint(s1, q_prev, 2 * (s1.q - qt), np.zeros_like(qt))
    g0 = free.adjoint(s0, q_prev, 2 * (s0.q - qt), np.zeros_like(qt))
    assert rel(g1["dL_dq_prev"], g0["dL_dq_prev"]) < 1e-6
    assert rel(g1["dL_dE"], g0["dL_dE"]) < 1e-6


# ---- points inside tets (barycentric weights) -------------------------------------------------

def _bary_case(k, compliance, shift=1e-3):
    """Cube-drop step k with points inside the four highest tets attached to targets lifted by
    ``shift`` (seeded barycentric weights)."""
    pb, q_prev, v_prev = rollout("cube_drop", k)
    sc = pb.scene
    cz = sc.X[sc.tets].mean(axis=1)[:, 2]
    tet_ids = np.argsort(-cz)[:4]
    tets = sc.tets[tet_ids]
    w = np.random.default_rng(7).dirichlet(np.ones(4), size=4)
    pts = np.einsum("bk,bkj->bj", w, q_prev[tets])
    bd = Bindings(tets, np.full(4, compliance), pts + np.array([0.0, 0.0, shift]), weight=w)
    bd.tet_ids = tet_ids  # the tets the points lie in (the GPU takes tet ids and weights)
    ct = sc.contacts(q_prev)
    st = Step(sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h, sc.gravity, ct, sc.eps, "neo_hookean", bd)
    return pb, st, bd, q_prev, v_prev


def test_unit_weights_reduce_to_the_single_vertex_binding():
    pb, st, bd, q_prev, v_prev = _case(2, 1e-4)
    n = st.mesh.n_verts
    others = np.stack([bd.vertex, (bd.vertex + 1) % n, (bd.vertex + 2) % n, (bd.vertex + 3) % n], axis=1)
    w = np.zeros((4, 4))
    w[:, 0] = 1.0
    b4 = Bindings(others, bd.compliance, bd.target, weight=w)
    q = q_prev + 1e-3
    z = np.random.default_rng(5).normal(size=q.shape)
    assert np.array_equal(b4.residual_term(q, st.h, n), bd.residual_term(q, st.h, n))
    assert abs(b4.matrix_term(st.h, n) - bd.matrix_term(st.h, n)).max() == 0.0
    for key, val in b4.gradients(q, z, st.h).items():
        assert np.array_equal(val, bd.gradients(q, z, st.h)[key])


def test_matrix_term_equals_the_stacked_rows_product():
    """h^2 J_b^T E_b^{-1} J_b from the coordinate triplets equals the product of the stacked rows."""
    pb, st, bd, q_prev, v_prev = _bary_case(0, 1e-4)
    n = st.mesh.n_verts
    Nm = bd.rows(n)
    dense = st.h ** 2 * Nm.T @ np.kron(np.diag(1.0 / bd.compliance), np.eye(3)) @ Nm
    assert np.allclose(bd.matrix_term(st.h, n).toarray(), dense, rtol=0, atol=1e-14 * np.abs(dense).max())
    q = q_prev + 1e-3
    assert np.allclose(bd.point(q), (Nm @ q.reshape(-1)).reshape(-1, 3))


@pytest.mark.parametrize("k", [0, 2])
def test_barycentric_gradients_match_central_differences(k):
    pb, st, bd, q_prev, v_prev = _bary_case(k, 1e-4)
    qt = pb.q_target
    base = st.forward(q_prev, v_prev)
    assert base.residual < 1e-9
    g = st.adjoint(base, q_prev, 2 * (base.q - qt), np.zeros_like(qt))

    def L(target=bd.target, compliance=bd.compliance):
        b2 = Bindings(bd.vertex, compliance, target, weight=bd.weight)
        s2 = Step(st.mesh.X, st.mesh.tets, st.E, st.nu, st.density, st.h, st.gravity, st.ct, st.eps, st.model, b2)
        r = s2.forward(q_prev, v_prev, q_init=base.q)
        assert r.residual < 1e-9
        return np.sum((r.q - qt) ** 2)

    d = np.random.default_rng(13).standard_normal(bd.target.shape)
    d /= np.linalg.norm(d)
    fd = (L(target=bd.target + 1e-7 * d) - L(target=bd.target - 1e-7 * d)) / 2e-7
    assert rel(np.sum(g["dL_dbinding_target"] * d), fd) < 1e-5
    e = 1e-4 * bd.compliance[0]
    de = np.zeros(bd.n)
    de[0] = 1.0
    fd = (L(compliance=bd.compliance + e * de) - L(compliance=bd.compliance - e * de)) / (2 * e)
    assert rel(g["dL_dcompliance"][0], fd) < 1e-5


def test_stiff_barycentric_bindings_converge_to_the_hard_attachment():
    """As for single vertices; a point inside a tet spreads the spring over four vertices (weights
    ~1/4), so the O(E_b) regime starts a decade stiffer."""
    errs_q, errs_g = [], []
    hard = None
    for E in (1e-5, 1e-6, 1e-7, 1e-8):
        pb, st, bd, q_prev, v_prev = _bary_case(0, E)
        assert st.nc == 0
        qt = pb.q_target
        s = st.forward(q_prev, v_prev, tol=1e-12)
        g = st.adjoint(s, q_prev, 2 * (s.q - qt), np.zeros_like(qt))
        if hard is None:
            Nm = bd.rows(st.mesh.n_verts)
            q_h, _ = constrained_step(st, q_prev, v_prev, s.q, Nm=Nm, d=bd.target)
            assert np.allclose(bd.point(q_h), bd.target, atol=1e-14)
            _, w_l = constrained_adjoint(st, q_h, q_prev, 2 * (q_h - qt), Nm=Nm, with_multiplier=True)
            hard = (q_h, w_l.reshape(-1, 3))
        errs_q.append(rel(s.q - q_prev, hard[0] - q_prev))
        errs_g.append(rel(g["dL_dbinding_target"], hard[1]))
    for e in (errs_q, errs_g):
        assert all(e[i + 1] < e[i] / 8 for i in range(len(e) - 1)), e
    assert errs_q[-1] < 1e-4 and errs_g[-1] < 1e-4, (errs_q, errs_g)


def test_models_bindings_and_friction_compose():
    """Co-rotational tets, stiff bindings and frictional contacts in one step: every gradient
    against central differences of the whole step."""
    pb, st0, bd, q_prev, v_prev = _case(2, 1e-5)
    sc = pb.scene
    mk = lambda E=sc.E, target=bd.target, compliance=bd.compliance: Step(  # noqa: E731
        sc.X, sc.tets, E, sc.nu, sc.density, sc.h, sc.gravity, st0.ct, sc.eps, "corotational",
        Bindings(bd.vertex, compliance, target))
    st = mk()
    qt = pb.q_target
    base = st.forward(q_prev, v_prev)
    assert base.residual < 1e-9 and st.nc > 0
    g = st.adjoint(base, q_prev, 2 * (base.q - qt), np.zeros_like(qt))

    def L(**kw):
        r = mk(**kw).forward(q_prev, v_prev, q_init=base.q)
        assert r.residual < 1e-9
        return np.sum((r.q - qt) ** 2)

    E0 = sc.E[0]
    fd = (L(E=E0 * (1 + 1e-6)) - L(E=E0 * (1 - 1e-6))) / (2e-6 * E0)
    assert rel(g["dL_dE"].sum(), fd) < 1e-5
    d = np.random.default_rng(17).standard_normal(bd.target.shape)
    d /= np.linalg.norm(d)
    fd = (L(target=bd.target + 1e-7 * d) - L(target=bd.target - 1e-7 * d)) / 2e-7
    assert rel(np.sum(g["dL_dbinding_target"] * d), fd) < 1e-5
    e = np.zeros(bd.n)
    e[1] = 1e-4 * bd.compliance[1]
    fd = (L(compliance=bd.compliance + e) - L(compliance=bd.compliance - e)) / (2 * e[1])
    assert rel(g["dL_dcompliance"][1], fd) < 1e-5
