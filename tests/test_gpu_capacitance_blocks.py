"""Capacitance solved iteratively: a scene whose contacts exceed the direct-inverse block size has
its full capacitance applied by an inner GMRES, preconditioned by exact inverses of groups of its
contacts, inside a flexible outer GMRES; and the capacitance inverted in FP32 inside an FP64
solve.  Both only change the preconditioner: the gradient must match the oracle as before."""
import pytest

torch = pytest.importorskip("torch")

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


@pytest.mark.parametrize("k", [2, 5])
@pytest.mark.parametrize("cap_block", [1, 4, 7, 13])
def test_split_capacitance_keeps_the_gradient(pkg, ctx, k, cap_block):
    case = step_case("cube_drop", k)
    nc = case[1].nc
    g0, ref, s0 = run_both(pkg, ctx, case, rtol=1e-12)
    g, ref, s = run_both(pkg, ctx, case, rtol=1e-12, cap_block=cap_block)
    assert s["capacitance_blocks"] == -(-nc // cap_block)
    assert s0["capacitance_blocks"] == 1 and s0["inner_iterations"] == 0
    assert s["rel_residual"] <= 1e-12
    assert_parity(g, ref, 1e-8, nc)
    if nc > cap_block:
        assert s["inner_iterations"] > 0
        # an inner solve to 1e-6 keeps the outer iteration count close to the direct inverse's
        assert s["iterations"] <= s0["iterations"] + 10, (s["iterations"], s0["iterations"])


def test_fp32_capacitance_in_an_fp64_solve(pkg, ctx):
    case = step_case("cube_drop", 5)
    g, ref, s = run_both(pkg, ctx, case, rtol=1e-12, cap_precision="mixed")
    assert s["rel_residual"] <= 1e-12
    assert_parity(g, ref, 1e-8, case[1].nc)
    g, ref, s = run_both(pkg, ctx, case, rtol=1e-8, cap_precision="mixed", cap_block=6)
    assert_parity(g, ref, 1e-5, case[1].nc)


def test_negative_cap_block_is_rejected(pkg, ctx):
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        run_both(pkg, ctx, step_case("cube_drop", 2), cap_block=-1)
