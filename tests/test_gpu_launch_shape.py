"""Launch shape of the A^{-1} product (chunks of 128, 256 or 512 nonzeros per warp) and the autotuner
that picks it: every chunk length gives the same products and gradients up to rounding, sizes other
than the three are rejected, and tune_adjoint runs on the GPU end to end (shape, then options)."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from tests._cases import rel, step_case  # noqa: E402
from tests.test_gpu_parity import KEYS, T, gpu_contacts, gpu_scene  # noqa: E402

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


def test_every_chunk_length_gives_the_same_products(pkg, ctx):
    """Beam (FP64 and FP32 products) and an uneven batch of blocks: A^{-1} x at 128 and 512 against 256."""
    import synth
    from paper_2603_16478_gb300.binding import elastic_solve
    sc = synth.beam_incline().scene
    beam = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    blocks = synth.block_batch(64)[:6]
    batch = pkg.Scene.batch(ctx, [(b.scene.X, b.scene.tets, b.scene.E, b.scene.nu, b.scene.density) for b in blocks],
                            blocks[0].scene.h)
    rng = np.random.default_rng(3)
    for scene in (beam, batch):
        x = torch.as_tensor(rng.normal(size=(scene.n_verts, 3)), device="cuda")
        ref = {p: elastic_solve(scene, x, precision=p).clone() for p in ("fp64", "mixed")}
        for n in (128, 512):
            scene.set_chunk(n)
            for p, tol in (("fp64", 1e-12), ("mixed", 1e-5)):
                e = (torch.linalg.norm(elastic_solve(scene, x, precision=p) - ref[p]) / torch.linalg.norm(ref[p])).item()
                assert e < tol, (scene.n_verts, n, p, e)
        scene.set_chunk(256)
        e = (torch.linalg.norm(elastic_solve(scene, x) - ref["fp64"]) / torch.linalg.norm(ref["fp64"])).item()
        assert e < 1e-14, e


def test_chunk_length_keeps_the_adjoint_gradients(pkg, ctx):
    """The cube after impact on one scene whose chunk length changes between calls: the FP64 adjoint
    gradients match the oracle at every length and agree with each other to rounding (the captured
    GMRES step graphs are rebuilt for the new chunk arrays)."""
    from tests.test_gpu_parity import assert_parity
    pb, st, s_, q_prev, v_prev = step_case("cube_drop", 5)
    sc = pb.scene
    rng = np.random.default_rng(0)
    dq = 2 * (s_.q - pb.q_target) + rng.normal(size=s_.q.shape) * 1e-4
    dv = rng.normal(size=s_.q.shape) * 1e-3
    ref = st.adjoint(s_, q_prev, dq, dv)
    scene = gpu_scene(pkg, ctx, sc)
    lam = s_.lam_frame(st, q_prev)
    outs = []
    side = torch.cuda.Stream()
    for n in (256, 512, 128, 256):
        scene.set_chunk(n)
        for stream in (None, side.cuda_stream):  # legacy stream (plain launches), then a captured-graph stream
            g, stats = pkg.adjoint_step(scene, gpu_contacts(pkg, st.ct), T(s_.q), T(q_prev), T(lam), T(dq), T(dv),
                                        eps=sc.eps, rtol=1e-12, stream=stream)
            torch.cuda.synchronize()
            assert_parity(g, ref, 1e-8, st.nc)
            outs.append(g)
    for g in outs[1:]:
        for k, _ in KEYS:
            assert rel(g[k].cpu().numpy(), outs[0][k].cpu().numpy()) < 1e-9, k


def test_unsupported_chunk_lengths_are_rejected(pkg, ctx):
    import synth
    sc = synth.beam_incline().scene
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    for n in (0, 100, 1024):
        with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
            scene.set_chunk(n)


def test_tune_adjoint_on_the_gpu(pkg, ctx):
    """The autotuner on the full-size beam at a GPU-forward state: it times the three chunk lengths
    and the option candidates, leaves the chosen chunk on the scene, and its choice reproduces the FP64
    gradients within the bound."""
    import synth
    from paper_2603_16478_gb300 import autotune as at
    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    scene = gpu_scene(pkg, ctx, sc)
    c = gpu_contacts(pkg, ct)
    q_prev, v_prev = T(pb.q0), T(pb.v0)
    q, lam, _ = pkg.forward_step(scene, c, q_prev, v_prev, None, tuple(sc.gravity), eps=sc.eps)
    dq = T(np.random.default_rng(4).normal(size=pb.q0.shape))
    cands = [{"precision": p, "cap_precision": cp, "restart": 64, "cap_block": 0}
             for p, cp in (("fp64", "fp64"), ("mixed", "mixed"), ("mixed", "tf32x3"), ("mixed", "refined"))]
    ch = at.tune_adjoint(scene, c, q, q_prev, lam.contiguous(), dq, None, eps=sc.eps, candidates=cands, repeats=2)
    assert ch.chunk in at.CHUNKS and scene.chunk == ch.chunk
    assert set(ch.chunk_ms) == set(at.CHUNKS) and all(np.isfinite(v) and v > 0 for v in ch.chunk_ms.values())
    assert all(t.error is None for t in ch.trials), [t.error for t in ch.trials]
    assert ch.rel_err <= 1e-3 and ch.options in cands
    g64, _ = pkg.adjoint_step(scene, c, q, q_prev, lam.contiguous(), dq, None, eps=sc.eps)
    g, _ = pkg.adjoint_step(scene, c, q, q_prev, lam.contiguous(), dq, None, eps=sc.eps,
                            precision=ch.options["precision"], cap_precision=ch.options["cap_precision"],
                            restart=ch.options["restart"])
    for k, _ in KEYS:
        assert rel(g[k].cpu().numpy(), g64[k].cpu().numpy()) <= 1e-3, k
