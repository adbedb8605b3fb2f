"""The allocation-free elastic solve (for callers that cannot have device memory allocated
during a call) gives the same result as the regular entry point, on two calls in a row.

Kept in a file that pytest collects last, so that a run stopping at the first failure has
already run every other test."""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

pytestmark = pytest.mark.gpu


def test_noalloc_elastic_solve_matches_regular_entry_point():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as pkg
    from paper_2603_16478_gb300.binding import elastic_solve_noalloc
    import synth

    pb = synth.beam_incline()
    sc = pb.scene
    ctx = pkg.Context(0)
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    rng = np.random.default_rng(7)
    y = torch.empty((sc.n_verts, 3), dtype=torch.float64, device="cuda")
    for _ in range(2):  # two calls in a row: the shared scratch must not carry anything over
        x = torch.as_tensor(rng.normal(size=(sc.n_verts, 3)), device="cuda")
        ref = pkg.elastic_solve(scene, x)
        elastic_solve_noalloc(scene, x, y)
        torch.cuda.synchronize()
        err = (torch.linalg.norm(y - ref) / torch.linalg.norm(ref)).item()
        assert err < 1e-12, err
    with pytest.raises(pkg.NcpadjError, match="INVALID_ARG"):
        elastic_solve_noalloc(scene, x, x)
