"""The large contact-heavy scene (ball pressed between the ground and a kinematic plate, 32
friction regions) on a down-scaled replica the oracle solves: GPU adjoint against the oracle in
FP64 and mixed precision, with the capacitance whole and split into blocks; gradients w.r.t.
per-vertex control forces and per-region friction."""
import functools

import numpy as np
import pytest

torch = pytest.importorskip("torch")

import synth  # noqa: E402
from tests._cases import make_step, rel  # noqa: E402
from tests.test_gpu_parity import T, gpu_contacts  # noqa: E402

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
def _case():
    pb = synth.sphere_press(cell=0.02)
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    st = make_step(sc, ct)
    s = st.forward(pb.q0, pb.v0)
    assert s.residual < 1e-8
    rng = np.random.default_rng(7)
    dq = 2 * (s.q - pb.q_target)
    ref = st.adjoint(s, pb.q0, dq, np.zeros_like(dq))
    return pb, st, s, dq, ref


@pytest.fixture(scope="module")
def scene(pkg, ctx):
    pb = _case()[0]
    sc = pb.scene
    return pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)


def _run(pkg, scene, **kw):
    pb, st, s, dq, ref = _case()
    lam = s.lam_frame(st, pb.q0)
    g, stats = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct), T(s.q), T(pb.q0), T(lam), T(dq), None,
                                eps=pb.scene.eps, **kw)
    return g, ref, stats


@pytest.mark.parametrize("cap_block", [0, 20])
def test_fp64_parity(pkg, scene, cap_block):
    g, ref, stats = _run(pkg, scene, rtol=1e-12, cap_block=cap_block)
    assert stats["rel_residual"] <= 1e-12
    assert stats["n_contacts"] == _case()[1].nc and _case()[1].ct.n_regions == 32
    for k, rk in (("dL_dfext", "dL_dfext"), ("dL_dmu", "dL_dmu_region"), ("dL_dq_prev", "dL_dq_prev"),
                  ("dL_dE", "dL_dE"), ("z", "z")):
        assert rel(g[k].cpu().numpy(), ref[rk]) <= 1e-8, (k, rel(g[k].cpu().numpy(), ref[rk]))


@pytest.mark.parametrize("cap_block", [0, 20])
def test_mixed_within_paper_tolerance(pkg, scene, cap_block):
    g, ref, stats = _run(pkg, scene, rtol=1e-8, precision="mixed", cap_precision="mixed", cap_block=cap_block)
    for k, rk in (("dL_dfext", "dL_dfext"), ("dL_dmu", "dL_dmu_region"), ("z", "z")):
        assert rel(g[k].cpu().numpy(), ref[rk]) <= 1e-3, (k, rel(g[k].cpu().numpy(), ref[rk]))


def test_woodbury_beats_jacobi_and_none(pkg, scene):
    its = {}
    for pc in ("woodbury", "jacobi", "none"):
        try:
            _, _, st = _run(pkg, scene, rtol=1e-8, precond=pc, max_iters=5000)
            its[pc] = st["iterations"]
        except pkg.NcpadjError as e:
            assert "NOT_CONVERGED" in str(e)
            its[pc] = 5001
    assert its["woodbury"] < its["jacobi"] and its["woodbury"] < its["none"], its
