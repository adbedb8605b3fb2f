"""One implicit time step: forward Newton solve and analytical adjoint by direct sparse LU.

Test infrastructure (oracle); see the package docstring.

Forward (Eq. dynamics, with p_i eliminated as the prox of G_i q and the contact multipliers
parametrised as in ``contact``):  unknowns q [3 n_v], lambda_n [n_c], gamma [n_c],
    R_q = M (q - qtilde) + h^2 sum_i w_i G_i^T (G_i q - p_i(q)) - h^2 sum_c J_c^T lambda_c
    R_n = FB_eps(delta_n, lambda_n),  R_f = FB_eps(||delta_f||, mu lambda_n - gamma)  (gamma = 0 if mu = 0)
    qtilde = qbar + h vbar + h^2 M^{-1} f_ext,  f_ext = M g + f_ctrl            (Sec. 3.1)
The multipliers are eliminated by the exact local solution of the contact equations and
the momentum residual is solved by damped Newton in q with a direct sparse LU.

Adjoint (Sec. 4.1):  script_A = A - Delta A + K_c,  with
    A - Delta A = M + h^2 sum_i w_i G_i^T (I - dp_i/dF) G_i,
    K_c         = h^2 sum_c J_c^T K_c J_c                       (Eq. final_diff_contact)
    script_A^T z = dL/dq + dL/dv / h                             (Eq. adjoint)
solved by a direct sparse LU of script_A^T.  Gradients (Eq. compute_gradient, App. B.3):
    dL/dqbar  = K_qbar^T z - dL/dv / h,   K_qbar = M + h^2 sum_c J_c^T K_c P_f J_c
    dL/dvbar  = h M z,   dL/dfext = h^2 z
    dL/dmu_c  = -h^2 (J_c z) . k_mu,c                             (summed per friction region)
    dL/dmu_i  = 2 h^2 V_i (G_i z) . (mu_i dp_i/dmu + p_i - G_i q)
    dL/dlam_i = 2 h^2 V_i mu_i (G_i z) . dp_i/dlam
    dL/dE_i, dL/dnu_i by the chain rule through mu(E, nu), lambda(E, nu).
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np
import scipy.sparse as sp
import scipy.sparse.linalg as spla

from . import contact as C
from .model import Mesh, lame, lame_derivatives
from . import models


@dataclass
class State:
    q: np.ndarray        # [n_v, 3]
    lam_n: np.ndarray    # [n_c]
    gamma: np.ndarray    # [n_c]
    residual: float = 0.0
    iterations: int = 0

    def lam_frame(self, step: "Step", q_prev):
        """lambda_c in frame coordinates [n_c, 3]."""
        out = np.zeros((len(self.lam_n), 3))
        for c in range(len(self.lam_n)):
            d = step.delta(self.q, q_prev, c)
            out[c] = C.contact_force(self.lam_n[c], self.gamma[c], d[1:])
        return out


class Step:
    """One time step of a scene with a frozen contact set."""

    def __init__(self, X, tets, E, nu, density, h, gravity, contacts, eps, model=models.NEO_HOOKEAN,
                 bindings=None, thickness=None, bend=0.0):
        # triangles (3 vertices per element) are shells of the given thickness (App. B.1, 2D formulation),
        # with isometric bending of stiffness `bend`
        tets = np.asarray(tets)
        if tets.shape[1] == 3:
            from .shell import TriMesh
            self.mesh = TriMesh(X, tets, 1e-3 if thickness is None else thickness)
            self.bend = float(bend)
            self.Qb = self.mesh.bending_matrix() if self.bend != 0.0 else None
        else:
            self.mesh = Mesh(X, tets)
            self.bend, self.Qb = 0.0, None
        models.by_model(model, self.mesh.n_tets)  # validates: one name, or one per tet
        self.model = model if isinstance(model, str) else np.asarray(model).copy()
        self.bindings = bindings  # oracle.binding.Bindings or None
        self.E = np.broadcast_to(np.asarray(E, float), (self.mesh.n_tets,)).copy()
        self.nu = np.broadcast_to(np.asarray(nu, float), (self.mesh.n_tets,)).copy()
        self.density = float(density)
        self.h = float(h)
        self.gravity = np.asarray(gravity, float)
        self.ct = contacts
        self.eps = float(eps)
        self.mass = self.mesh.lumped_mass(self.density)
        self.N = 3 * self.mesh.n_verts
        self.verbose = False

    # ---- helpers ------------------------------------------------------------------------
    @property
    def nc(self):
        return self.ct.n

    def lame(self):
        return lame(self.E, self.nu)

    def delta(self, q, q_prev, c):
        v = self.ct.vertex[c]
        Fc = self.ct.frame[c]
        dn = Fc[0] @ q[v] - self.ct.d_n[c]
        df = Fc[1:] @ (q[v] - q_prev[v]) - self.ct.d_f[c]
        return np.array([dn, df[0], df[1]])

    def qtilde(self, q_prev, v_prev, f_ctrl):
        f_ext = self.mass[:, None] * self.gravity[None, :] + f_ctrl
        return q_prev + self.h * v_prev + self.h * self.h * f_ext / self.mass[:, None]

    # ---- forward ------------------------------------------------------------------------
    def residual(self, q, lam_n, gam, q_prev, qt, mu_c=None):
        """[R_q / h^2, R_n, R_f] of Eq. (dynamics) with p_i = prox(G_i q)."""
        mu_c = self.ct.mu if mu_c is None else mu_c
        h2 = self.h * self.h
        mesh = self.mesh
        mu_L, lam_L = self.lame()
        F = mesh.F(q)
        P = models.prox(self.model, F, mu_L, lam_L)
        w = 2.0 * mu_L * mesh.vol
        r_el = np.einsum("tji,tj->ti", mesh.G, mesh.vec(F - P))
        Rq = (self.mass[:, None] * (q - qt)).reshape(-1) + h2 * mesh.scatter_vectors(w[:, None] * r_el)
        if self.Qb is not None:
            Rq = Rq + h2 * self.bend * (self.Qb @ q.reshape(-1))
        if self.bindings is not None:
            Rq = Rq + self.bindings.residual_term(q, self.h, mesh.n_verts)
        Rn = np.zeros(self.nc)
        Rf = np.zeros(self.nc)
        for c in range(self.nc):
            v = self.ct.vertex[c]
            d = self.delta(q, q_prev, c)
            _, nf = C.tangent_dir(d[1:])
            Rq[3 * v:3 * v + 3] -= h2 * self.ct.frame[c].T @ C.contact_force(lam_n[c], gam[c], d[1:])
            Rn[c] = C.fb(d[0], lam_n[c], self.eps)
            Rf[c] = C.fb(nf, mu_c[c] * lam_n[c] - gam[c], self.eps) if mu_c[c] > 0 else gam[c]
        return np.concatenate([Rq / h2, Rn, Rf])

    def local_multipliers(self, q, q_prev, mu_c=None):
        """(lambda_n, gamma) solving the contact equations exactly at q, or None if some
        contact has delta_n <= 0 or zero slip (outside the domain of the local solve)."""
        mu_c = self.ct.mu if mu_c is None else mu_c
        lam_n = np.zeros(self.nc)
        gam = np.zeros(self.nc)
        for c in range(self.nc):
            d = self.delta(q, q_prev, c)
            if d[0] <= 0 or (mu_c[c] > 0 and np.linalg.norm(d[1:]) == 0.0):
                return None
            lam_n[c], gam[c] = C.local_solve(d, mu_c[c], self.eps)
        return lam_n, gam

    def start_point(self, q_prev, qt, seed=0):
        """The inertial prediction (its slips point along the free motion), with every contact
        vertex lifted along its normal to a small positive gap.  If the prediction inverts a tet
        (large forces on light vertices), it is pulled back towards q_prev by halving
        q_prev + t (qt - q_prev) until no tet is inverted."""
        rng = np.random.default_rng(seed)
        q = qt.copy()
        t = 1.0
        while self.mesh.min_jacobian(self.mesh.F(q)) <= 0 and t > 1e-12:
            t *= 0.5
            q = q_prev + t * (qt - q_prev)
        gap0 = 10.0 * self.eps * self.eps / (np.max(self.mass) * np.linalg.norm(self.gravity) + 1e-300)
        for c in range(self.nc):
            v = self.ct.vertex[c]
            dn = self.delta(q, q_prev, c)[0]
            if dn < gap0:
                q[v] += (gap0 - dn) * self.ct.frame[c][0]
            if np.linalg.norm(self.delta(q, q_prev, c)[1:]) == 0.0:
                q[v] += 1e-12 * (self.ct.frame[c][1:].T @ rng.normal(size=2))
        return q

    def forward(self, q_prev, v_prev, f_ctrl=None, mu_c=None, q_init=None, tol=1e-9,
                       max_iter=200, seed=0):
        """Converged step by Newton in q alone (Returns State).

        The multipliers are eliminated through the exact local solution of the contact
        equations (lambda_n = eps^2/delta_n, gamma = mu lambda_n - eps^2/||delta_f||), so
        the iterate always satisfies them and only the momentum residual R_q(q) remains.
        Its Jacobian is the adjoint matrix script_A.  The line search keeps every contact
        inside the domain of the local solve (delta_n > 0, nonzero slip) and asks for a
        decrease of ||R_q||; it also refuses steps that turn the slip of a contact carrying a
        real friction force (gamma > 0.05 mu lambda_n) by more than 60 degrees, so the iterate
        stays on the branch connected to the inertial prediction (friction opposing the slip).  Stops at ||R_q||_inf <= tol * max_v(m_v |g|), or when
        no step decreases ||R_q|| any more once that tolerance is met (rounding floor).
        """
        q_prev = np.asarray(q_prev, float)
        f_ctrl = np.zeros_like(q_prev) if f_ctrl is None else f_ctrl
        qt = self.qtilde(q_prev, v_prev, f_ctrl)
        N = self.N
        q = self.start_point(q_prev, qt, seed) if q_init is None else q_init.copy()
        scale_f = np.max(self.mass) * np.linalg.norm(self.gravity) + 1e-300

        def resid(qq):
            lm = self.local_multipliers(qq, q_prev, mu_c) if self.nc else (np.zeros(0), np.zeros(0))
            if lm is None:
                return None, None
            R = self.residual(qq, lm[0], lm[1], q_prev, qt, mu_c)
            return R[:N], lm

        def slips(qq):
            return np.array([self.delta(qq, q_prev, c)[1:] for c in range(self.nc)]).reshape(-1, 2)

        R, lm = resid(q)
        it = 0
        for it in range(1, max_iter + 1):
            res = np.max(np.abs(R)) / scale_f
            st = State(q, lm[0], lm[1])
            Amat, _ = self.adjoint_matrix(st, q_prev, mu_c)
            dq = -spla.spsolve(Amat.tocsc(), R * self.h * self.h).reshape(-1, 3)
            t = 1.0
            phi0 = R @ R
            s0 = slips(q)
            mu_now = self.ct.mu if mu_c is None else mu_c
            loaded = lm[1] > 0.05 * mu_now * lm[0]  # the turn rule guards contacts with real friction
            accepted = False
            for _ in range(40):
                qn = q + t * dq
                s1 = slips(qn)
                cosines_ok = np.sum(s0 * s1, axis=1) >= 0.5 * np.linalg.norm(s0, axis=1) * np.linalg.norm(s1, axis=1)
                turn_ok = np.all(cosines_ok | ~loaded)
                if turn_ok:
                    try:
                        Rn, lmn = resid(qn)
                    except ValueError:
                        Rn = None
                    if Rn is not None and Rn @ Rn <= (1 - 1e-4 * t) * phi0:
                        accepted = True
                        break
                t *= 0.5
            if not accepted:
                break  # no decrease possible: rounding floor (or a failure, reported via residual)
            q, R, lm = qn, Rn, lmn
            if np.max(np.abs(R)) / scale_f <= tol * 1e-2:
                break
            if self.verbose:
                print(f"  it={it} res={np.max(np.abs(R)) / scale_f:.3e} t={t:.3g}")
        return State(q, lm[0], lm[1], np.max(np.abs(R)) / scale_f, it)

    # ---- adjoint ------------------------------------------------------------------------
    def contact_blocks(self, state: State, q_prev, mu_c=None, eps=None):
        """Per contact K_c (frame coords) and k_mu, via implicit differentiation."""
        mu_c = self.ct.mu if mu_c is None else mu_c
        eps = self.eps if eps is None else eps
        K = np.zeros((self.nc, 3, 3))
        kmu = np.zeros((self.nc, 3))
        for c in range(self.nc):
            d = self.delta(state.q, q_prev, c)
            K[c], kmu[c] = C.contact_jacobians(d, state.lam_n[c], state.gamma[c], mu_c[c], eps)
        return K, kmu

    def adjoint_matrix(self, state: State, q_prev, mu_c=None, eps=None):
        """(script_A, pieces) with script_A the sparse adjoint matrix (not transposed)."""
        mesh = self.mesh
        h2 = self.h * self.h
        mu_L, lam_L = self.lame()
        F = mesh.F(state.q)
        P = models.prox(self.model, F, mu_L, lam_L)
        Jp, dP_dmu, dP_dlam = models.prox_derivatives(self.model, F, P, mu_L, lam_L)
        w = 2.0 * mu_L * mesh.vol
        blocks = h2 * w[:, None, None] * np.einsum("tki,tkl,tlj->tij", mesh.G, np.eye(mesh.nF) - Jp, mesh.G)
        A_el = sp.diags(np.repeat(self.mass, 3)) + mesh.scatter_blocks(blocks)
        if self.Qb is not None:
            A_el = A_el + h2 * self.bend * self.Qb
        if self.bindings is not None:
            A_el = A_el + self.bindings.matrix_term(self.h, mesh.n_verts)
        K, kmu = self.contact_blocks(state, q_prev, mu_c, eps)
        rows, cols, vals = [], [], []
        for c in range(self.nc):
            v = self.ct.vertex[c]
            Fc = self.ct.frame[c]
            blk = h2 * Fc.T @ K[c] @ Fc
            for a in range(3):
                for b in range(3):
                    rows.append(3 * v + a); cols.append(3 * v + b); vals.append(blk[a, b])
        Kc = sp.coo_matrix((vals, (rows, cols)), shape=(self.N, self.N)).tocsr()
        pieces = dict(F=F, P=P, Jp=Jp, dP_dmu=dP_dmu, dP_dlam=dP_dlam, K=K, kmu=kmu, A_el=A_el, Kc=Kc,
                      mu_L=mu_L, lam_L=lam_L)
        return (A_el + Kc).tocsr(), pieces

    def adjoint(self, state: State, q_prev, dL_dq, dL_dv, mu_c=None, eps=None):
        """All one-step gradients for seeds dL/dq, dL/dv [n_v, 3]: z from a direct sparse LU of
        script_A^T z = dL/dq + dL/dv / h (Eq. adjoint), then the contractions.  Returns dict."""
        Amat, pc = self.adjoint_matrix(state, q_prev, mu_c, eps)
        b = (np.asarray(dL_dq) + np.asarray(dL_dv) / self.h).reshape(-1)
        z = spla.spsolve(Amat.T.tocsc(), b)
        out = self.contract(state, z, dL_dv, pc)
        out["A"] = Amat
        return out

    def contract(self, state: State, z, dL_dv, pc):
        """The gradients of Eq. (compute_gradient) for a given adjoint solution z [3 n_v] (pieces
        ``pc`` from adjoint_matrix at the same state)."""
        mesh = self.mesh
        h = self.h
        h2 = h * h
        z = np.asarray(z, float).reshape(-1)
        out = dict(z=z.reshape(-1, 3))
        # K_qbar = M + h^2 sum_c J_c^T K_c P_f J_c
        Pf = np.diag([0.0, 1.0, 1.0])
        gq = np.repeat(self.mass, 3) * z
        gq = gq.reshape(-1, 3)
        dmu_c = np.zeros(self.nc)
        for c in range(self.nc):
            v = self.ct.vertex[c]
            Fc = self.ct.frame[c]
            Kq = h2 * Fc.T @ pc["K"][c] @ Pf @ Fc
            gq[v] += Kq.T @ z.reshape(-1, 3)[v]
            dmu_c[c] = -h2 * (Fc @ z.reshape(-1, 3)[v]) @ pc["kmu"][c]
        out["dL_dq_prev"] = gq - np.asarray(dL_dv) / h
        out["dL_dv_prev"] = h * self.mass[:, None] * z.reshape(-1, 3)
        out["dL_dfext"] = h2 * z.reshape(-1, 3)
        out["dL_dmu_contact"] = dmu_c
        nreg = self.ct.n_regions
        out["dL_dmu_region"] = np.bincount(self.ct.region, weights=dmu_c, minlength=nreg) if self.nc else np.zeros(nreg)
        # elastic parameters
        vec = mesh.vec
        Gz = mesh.Gx(z)                       # vec(G_i z)  [n_t, 9] ([n_t, 6] for triangles)
        mu_L, lam_L = pc["mu_L"], pc["lam_L"]
        pmF = vec(pc["P"] - pc["F"])
        dmu = 2.0 * h2 * mesh.vol * np.sum(Gz * (mu_L[:, None] * vec(pc["dP_dmu"]) + pmF), axis=1)
        dlam = 2.0 * h2 * mesh.vol * mu_L * np.sum(Gz * vec(pc["dP_dlam"]), axis=1)
        dmu_dE, dlam_dE, dmu_dnu, dlam_dnu = lame_derivatives(self.E, self.nu)
        out["dL_dmuL"] = dmu
        out["dL_dlamL"] = dlam
        out["dL_dE"] = dmu * dmu_dE + dlam * dlam_dE
        out["dL_dnu"] = dmu * dmu_dnu + dlam * dlam_dnu
        if self.Qb is not None:  # the bending force h^2 k_b Q q of the residual
            out["dL_dbend"] = -h2 * float(z @ (self.Qb @ state.q.reshape(-1)))
        if self.bindings is not None:
            out.update(self.bindings.gradients(state.q, z, h))
        return out
