"""Bilateral bindings on single vertices (Eq. binding) on the GPU against the FP64 oracle: adjoint
parity of every gradient including dL/dd_b and dL/dE_b, with and without contacts and with a
stiff compliance; mixed precision; the forward step's converged state; argument errors."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import rel  # noqa: E402
from tests.test_gpu_parity import KEYS, T, gpu_contacts, gpu_scene  # noqa: E402
from tests.test_oracle_bindings import _case  # noqa: E402

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


@functools.lru_cache(maxsize=None)
def _oracle(k, compliance):
    pb, st, bd, q_prev, v_prev = _case(k, compliance)
    s = st.forward(q_prev, v_prev, tol=1e-12)
    assert s.residual < 1e-9
    return pb, st, bd, q_prev, v_prev, s


def _gpu_bindings(pkg, bd):
    return pkg.Bindings(T(bd.vertex, torch.int32), T(bd.target), T(bd.compliance))


def _adjoint(pkg, ctx, k, compliance, rtol, **kw):
    pb, st, bd, q_prev, v_prev, s = _oracle(k, compliance)
    rng = np.random.default_rng(4)
    dq = 2 * (s.q - pb.q_target) + rng.normal(size=s.q.shape) * 1e-4
    dv = rng.normal(size=s.q.shape) * 1e-3
    ref = st.adjoint(s, q_prev, dq, dv)
    scene = gpu_scene(pkg, ctx, pb.scene)
    lam = s.lam_frame(st, q_prev) if st.nc else np.zeros((0, 3))
    g, stats = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct), T(s.q), T(q_prev), T(lam), T(dq), T(dv),
                                eps=pb.scene.eps, rtol=rtol, bindings=_gpu_bindings(pkg, bd), **kw)
    torch.cuda.synchronize()
    errs = {}
    for key, rk in KEYS + [("dL_dbinding_target", "dL_dbinding_target"), ("dL_dcompliance", "dL_dcompliance")]:
        if st.nc == 0 and key in ("dL_dmu", "dL_dmu_contact"):
            continue
        errs[key] = rel(g[key].cpu().numpy().reshape(-1), np.asarray(ref[rk]).reshape(-1))
    return stats, errs


@pytest.mark.parametrize("k,compliance", [(0, 1e-4), (2, 1e-4), (5, 1e-4), (0, 1e-7)])
def test_adjoint_parity(pkg, ctx, k, compliance):
    stats, errs = _adjoint(pkg, ctx, k, compliance, rtol=1e-12)
    assert stats["rel_residual"] <= 1e-12
    assert max(errs.values()) <= 1e-8, errs


@pytest.mark.parametrize("k", [0, 2])
def test_adjoint_mixed_precision(pkg, ctx, k):
    _, errs = _adjoint(pkg, ctx, k, 1e-4, rtol=1e-8, precision="mixed", cap_precision="mixed")
    assert max(errs.values()) <= 1e-3, errs


@pytest.mark.parametrize("k", [0, 2, 5])
def test_forward_matches_oracle_state(pkg, ctx, k):
    pb, st, bd, q_prev, v_prev, s = _oracle(k, 1e-4)
    sc = pb.scene
    q, lam, stats = pkg.forward_step(gpu_scene(pkg, ctx, sc), gpu_contacts(pkg, st.ct), T(q_prev), T(v_prev), None,
                                     tuple(sc.gravity), eps=sc.eps, newton_tol=1e-11, max_newton=200,
                                     bindings=_gpu_bindings(pkg, bd))
    assert stats["residual"] < 1e-8
    assert rel(q.cpu().numpy() - q_prev, s.q - q_prev) < 1e-7
    if st.nc:
        assert rel(lam.cpu().numpy(), s.lam_frame(st, q_prev)) < 1e-6


def test_invalid_bindings_are_rejected(pkg, ctx):
    pb, st, bd, q_prev, v_prev, s = _oracle(0, 1e-4)
    scene = gpu_scene(pkg, ctx, pb.scene)
    dq = T(2 * (s.q - pb.q_target))

    def call(vertex, compliance, **kw):
        b = pkg.Bindings(T(vertex, torch.int32), T(bd.target), T(compliance))
        return pkg.adjoint_step(scene, None, T(s.q), T(q_prev), T(np.zeros((0, 3))), dq, None, eps=pb.scene.eps,
                                bindings=b, **kw)

    bad_v = bd.vertex.copy()
    bad_v[2] = scene.n_verts
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        call(bad_v, bd.compliance)
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        call(bd.vertex, np.array([1e-4, 0.0, 1e-4, 1e-4]))
    # the scene still works after the rejected calls
    g, stats = call(bd.vertex, bd.compliance, rtol=1e-10)
    assert stats["rel_residual"] <= 1e-10
    assert torch.isfinite(g["dL_dcompliance"]).all()


@pytest.mark.parametrize("k", [2, 5])
def test_stiff_bindings_are_preconditioned_exactly(pkg, ctx, k):
    """The bindings sit in the Woodbury low-rank term beside the contacts (Sec. 3.2.1, Sec. 4.4): the
    capacitance counts their rows, and stiff springs (E_b = 1e-7) cost no more Krylov iterations
    than soft ones (E_b = 1e-4) -- left out of the preconditioner they cost up to 3 n_b more."""
    st_soft, errs = _adjoint(pkg, ctx, k, 1e-4, rtol=1e-10)
    assert max(errs.values()) <= 1e-6, errs
    st_stiff, errs = _adjoint(pkg, ctx, k, 1e-7, rtol=1e-10)
    assert max(errs.values()) <= 1e-6, errs
    nb = len(_case(k, 1e-7)[2].vertex)
    nc = _oracle(k, 1e-7)[1].nc
    assert st_stiff["capacitance_dim"] == 3 * (nc + nb)
    assert st_stiff["iterations"] <= st_soft["iterations"] + 3, (st_stiff["iterations"], st_soft["iterations"])
    _, errs = _adjoint(pkg, ctx, k, 1e-7, rtol=1e-10, cap_drop=0.0)  # every member kept: same gradients
    assert max(errs.values()) <= 1e-6, errs
