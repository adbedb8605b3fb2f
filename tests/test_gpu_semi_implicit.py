"""The semi-implicit fixed-point baseline on the GPU (NCPADJ_SOLVER_SEMI_IMPLICIT with the elastic
preconditioner, Sec. 4.4 Eq. semi-implicit) against the oracle's iteration: contact-free it takes
the oracle's number of iterations to the same tolerance and gives the oracle's gradients; resting
on contacts both diverge, and the GPU says so (NOT_CONVERGED) instead of returning a gradient,
while Woodbury-preconditioned GMRES solves the same system."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from oracle.semi_implicit import elastic_part, semi_implicit  # noqa: E402
from tests._cases import step_case  # noqa: E402
from tests.test_gpu_parity import assert_parity, run_both  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


@pytest.fixture(scope="module")
def ctx(pkg):
    return pkg.Context(0)


def _oracle_iterations(case, seed, rtol):
    pb, st, s, q_prev, v_prev = case
    rng = np.random.default_rng(seed)
    dq = 2 * (s.q - pb.q_target) + rng.normal(size=s.q.shape) * 1e-4
    dv = rng.normal(size=s.q.shape) * 1e-3
    Aadj, _ = st.adjoint_matrix(s, q_prev)
    b = (dq + dv / pb.scene.h).reshape(-1)
    _, hist, ok = semi_implicit(elastic_part(st), Aadj.T.tocsr(), b, rtol=rtol, max_iters=3000)
    return len(hist) - 1, ok


def test_contact_free_semi_implicit_matches_the_oracle(pkg, ctx):
    case = step_case("cube_drop", 0)
    assert case[1].nc == 0
    its, ok = _oracle_iterations(case, 0, 1e-9)
    assert ok
    g, ref, stats = run_both(pkg, ctx, case, seed=0, rtol=1e-9, solver="semi_implicit", precond="elastic",
                             max_iters=3000)
    assert stats["solver_used"] == 4
    assert abs(stats["iterations"] - its) <= 1, (stats["iterations"], its)
    assert_parity(g, ref, 1e-6, 0)


def test_resting_contacts_make_both_diverge(pkg, ctx):
    case = step_case("cube_drop", 5)
    its, ok = _oracle_iterations(case, 1, 1e-8)
    assert not ok and its <= 5
    with pytest.raises(pkg.NcpadjError, match="NOT_CONVERGED") as e:
        run_both(pkg, ctx, case, seed=1, rtol=1e-8, solver="semi_implicit", precond="elastic", max_iters=3000)
    assert e.value.stats["iterations"] <= 5 and e.value.stats["rel_residual"] > 1.0
    g, ref, stats = run_both(pkg, ctx, case, seed=1, rtol=1e-12)  # the Krylov solve of the same system
    assert_parity(g, ref, 1e-8, case[1].nc)
