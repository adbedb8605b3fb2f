"""The semi-implicit fixed-point baseline of the adjoint solve (test infrastructure, oracle).

Sec. 4.4 (Eq. semi-implicit): earlier projective-dynamics frameworks solve the linear adjoint
system by reusing the forward solver's local-global split, i.e. the stationary iteration

    A z^{k+1} = (A - B) z^k + b,       B = script_A^T,  A = M + h^2 sum_i w_i G_i^T G_i,

which treats the constant elastic matrix A implicitly and the rest of B explicitly.  It converges
exactly when the spectral radius of A^{-1}(A - B) is below 1.  The paper's solver study (Sec. 5)
takes it as the baseline against which the preconditioned Krylov methods are measured.

Written here from that equation: a sparse LU of A, then the iteration, with z^0 = 0.
"""
from __future__ import annotations

import numpy as np
import scipy.sparse.linalg as spla

from .model import elastic_matrix


def elastic_part(step):
    """A = M + h^2 sum_i w_i G_i^T G_i of a Step (Eq. dynamics), sparse [3 n_v, 3 n_v]; a shell's
    constant bending Hessian h^2 k_b Q belongs to it too."""
    mu_L, _ = step.lame()
    A = elastic_matrix(step.mesh, step.mass, mu_L, step.h)
    if getattr(step, "Qb", None) is not None:
        A = A + step.h * step.h * step.bend * step.Qb
    return A.tocsc()


def semi_implicit(A, B, b, rtol=1e-10, max_iters=1000, blowup=1e6):
    """Iterate A z^{k+1} = (A - B) z^k + b from z^0 = 0.

    Returns (z, residual history [||b - B z^k|| / ||b|| for k = 0, 1, ...], converged).  Stops at
    rtol, after max_iters, or once the residual exceeds blowup (divergence)."""
    lu = spla.splu(A.tocsc())
    b = np.asarray(b, float).reshape(-1)
    bn = np.linalg.norm(b)
    z = np.zeros_like(b)
    hist = [1.0]
    if bn == 0.0:
        return z, hist, True
    for _ in range(max_iters):
        z = lu.solve((A @ z) - (B @ z) + b)
        r = np.linalg.norm(b - B @ z) / bn
        hist.append(r)
        if not np.isfinite(r) or r <= rtol or r > blowup:
            break
    return z, hist, bool(hist[-1] <= rtol)


def spectral_radius(A, B):
    """rho(A^{-1}(A - B)) by a dense eigenvalue decomposition (tiny meshes only)."""
    Ad = A.toarray()
    Bd = B.toarray()
    return float(np.max(np.abs(np.linalg.eigvals(np.linalg.solve(Ad, Ad - Bd)))))
