"""Pins of the oracle's semi-implicit fixed-point baseline (Sec. 4.4, Eq. semi-implicit):

* the k-th iterate equals the partial Neumann sum sum_{i<k} T^i A^{-1} b, T = A^{-1}(A - B), formed
  from dense matrix powers (closed form of the stationary iteration);
* contact-free, rho(T) < 1: the residual contracts asymptotically at rate rho(T) and the iterate
  reaches the direct solution;
* resting on contacts, rho(T) >> 1 (the contact stiffness lives only in B): the iteration
  diverges -- the failure the paper's solver study shows for this baseline.
"""
import numpy as np

from oracle.semi_implicit import elastic_part, semi_implicit, spectral_radius
from tests._cases import step_case


def _system(k):
    pb, st, s, q_prev, v_prev = step_case("cube_drop", k)
    Aadj, _ = st.adjoint_matrix(s, q_prev)
    return elastic_part(st), Aadj.T.tocsr(), st


def test_iterates_are_the_partial_neumann_sums():
    A, B, _ = _system(1)
    b = np.random.default_rng(0).normal(size=B.shape[0])
    Ad, Bd = A.toarray(), B.toarray()
    T = np.linalg.solve(Ad, Ad - Bd)
    c = np.linalg.solve(Ad, b)
    ref, term = np.zeros_like(b), c.copy()
    for k in range(1, 6):
        ref = ref + term
        term = T @ term
        z, hist, _ = semi_implicit(A, B, b, rtol=0.0, max_iters=k)
        assert len(hist) == k + 1
        assert np.linalg.norm(z - ref) <= 1e-12 * np.linalg.norm(ref)


def test_contact_free_iteration_contracts_at_the_spectral_radius_and_converges():
    A, B, st = _system(0)
    assert st.nc == 0
    rho = spectral_radius(A, B)
    assert 0.5 < rho < 1.0
    b = np.random.default_rng(1).normal(size=B.shape[0])
    z, hist, ok = semi_implicit(A, B, b, rtol=1e-11, max_iters=2000)
    assert ok
    rates = np.array(hist[-50:]) / np.array(hist[-51:-1])
    assert abs(np.median(rates) - rho) < 2e-3 * rho
    import scipy.sparse.linalg as spla
    zd = spla.spsolve(B.tocsc(), b)
    assert np.linalg.norm(z - zd) <= 1e-8 * np.linalg.norm(zd)


def test_resting_contacts_make_it_diverge():
    A, B, st = _system(5)
    assert st.nc > 0
    assert spectral_radius(A, B) > 1e3
    b = np.random.default_rng(2).normal(size=B.shape[0])
    _, hist, ok = semi_implicit(A, B, b, rtol=1e-10, max_iters=50)
    assert not ok and hist[-1] > 1e6
