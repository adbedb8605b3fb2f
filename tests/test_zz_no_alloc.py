"""The allocation-free elastic solve gives the same result as the regular entry point, on two calls
in a row, and allocates no device memory while it runs.

It is for callers that cannot have device memory allocated during a call: programs whose device
memory is reserved up front by their own pool, and loops with hard latency limits.  Kept in a
file that pytest collects last, so that a run stopping at the first failure has already run
every other test; it passes alone in a fresh process as well."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def pkg():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as p
    return p


def test_noalloc_elastic_solve_matches_regular_entry_point_and_allocates_nothing(pkg):
    from paper_2603_16478_gb300.binding import elastic_solve_noalloc
    import synth

    pb = synth.beam_incline()
    sc = pb.scene
    ctx = pkg.Context(0)
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    rng = np.random.default_rng(7)
    y = torch.empty((sc.n_verts, 3), dtype=torch.float64, device="cuda")
    xs = [torch.as_tensor(rng.normal(size=(sc.n_verts, 3)), device="cuda") for _ in range(2)]
    refs = [pkg.elastic_solve(scene, x) for x in xs]  # loads the kernels both entry points use
    torch.cuda.synchronize()
    for x, ref in zip(xs, refs):  # the first call after the context's creation, then a second one
        free0 = torch.cuda.mem_get_info()[0]
        elastic_solve_noalloc(scene, x, y)
        torch.cuda.synchronize()
        assert torch.cuda.mem_get_info()[0] == free0  # no device memory taken by the call
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-12, err  # the shared scratch carries nothing over from the previous call
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        elastic_solve_noalloc(scene, xs[0], xs[0])  # aliased
    with pytest.raises(ValueError):
        elastic_solve_noalloc(scene, xs[0], y.float())  # y must be float64 of the scene's shape


def test_noalloc_rejects_scenes_above_its_limit(pkg):
    """More than 262,144 vertices (here a batch of 65 blocks of 16^3 vertices) is INVALID_ARG."""
    from paper_2603_16478_gb300.binding import elastic_solve_noalloc
    import synth

    X, tets = synth.hex_tet_mesh(15, 15, 15, 0.01)
    n = 65
    assert n * X.shape[0] > 262144
    ctx = pkg.Context(0)
    scene = pkg.Scene.batch(ctx, [(X, tets, 1e5, 0.4, 1000.0)] * n, 1.0 / 60)
    x = torch.zeros((scene.n_verts, 3), dtype=torch.float64, device="cuda")
    y = torch.empty_like(x)
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        elastic_solve_noalloc(scene, x, y)
