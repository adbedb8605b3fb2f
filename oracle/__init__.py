"""FP64 CPU oracle for the one-step analytical adjoint (test infrastructure only).

This package is the slow, plain reference that the CUDA path is checked against.  Only
``tests/``, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline / reference arm may
import it; the product path (``paper_2603_16478_gb300``) never does, and the two share no
code besides the seeded input generators in ``synth``.

Where the method has a plain definition, the oracle writes that definition out instead of
the paper's fast route:

* the Neo-Hookean prox p(F) is a 9-D Newton minimisation of mu||P-F||^2 + zeta(P) with
  invariant-based derivatives (no SVD),
* the co-rotational and ARAP projections (App. B.2) come from the polar decomposition F = R S
  and its differential (``models``),
* its Jacobian dp/dF is the implicit-function-theorem form (I + grad^2 zeta / w)^{-1}
  of Eq. (pd_expanded), and dp/dmu, dp/dlambda likewise,
* the contact Jacobian K_c = -d lambda_c / d delta_c comes from implicit differentiation of
  the smoothed Fischer-Burmeister residuals of Eq. (contact) (exact partials),
* the adjoint matrix is assembled explicitly and solved by a direct sparse LU (no
  preconditioner, no Krylov method),
* the forward step is a plain damped Newton method on the coupled residual of
  Eq. (dynamics), used for finite-difference checks of the whole gradient.

The paper's SVD closed form of the projection Jacobian (Sec. 4.3, App. B) is also written
out here (``paper_svd``) so that its readings can be pinned on the CPU before any kernel
uses them.
"""
