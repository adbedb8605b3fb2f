"""The seeded input generators shared by the oracle, the GPU tests and the bench (CPU only):
the same seed gives the same bytes, meshes are valid, contact sets are well-formed, and the
workloads have the sizes their recipe states."""
import numpy as np
import pytest

import synth

GENERATORS = {
    "cube": lambda seed: synth.cube_drop(seed=seed),
    "beam": lambda seed: synth.beam_incline(seed=seed),
    "two_tet": lambda seed: synth.two_tet(seed=seed),
    "ball_replica": lambda seed: synth.sphere_press(seed=seed, cell=0.02),
}


def _arrays(pb):
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    return [sc.X, sc.tets, np.asarray(sc.E), np.asarray(sc.nu), pb.q0, pb.v0, pb.q_target, ct.vertex, ct.frame,
            ct.d_n, ct.mu, ct.region]


@pytest.mark.parametrize("name", sorted(GENERATORS))
def test_same_seed_same_bytes(name):
    a, b = _arrays(GENERATORS[name](0)), _arrays(GENERATORS[name](0))
    for x, y in zip(a, b):
        assert np.asarray(x).tobytes() == np.asarray(y).tobytes()


@pytest.mark.parametrize("name", sorted(GENERATORS))
def test_meshes_and_contacts_are_well_formed(name):
    pb = GENERATORS[name](0)
    sc = pb.scene
    X, T = sc.X, sc.tets
    e = X[T[:, 1:]] - X[T[:, [0]]]
    vol = np.einsum("ij,ij->i", np.cross(e[:, 0], e[:, 1]), e[:, 2]) / 6.0
    assert vol.min() > 0  # positively oriented, none degenerate
    assert np.array_equal(np.unique(T), np.arange(len(X)))  # every vertex in some tet
    ct = sc.contacts(pb.q0)
    if ct.n:
        F = ct.frame
        assert np.allclose(np.einsum("cij,ckj->cik", F, F), np.eye(3), atol=1e-12)  # orthonormal rows
        assert np.all(np.linalg.det(F) > 0)
        assert len(np.unique(ct.vertex)) == ct.n and ct.vertex.max() < len(X)
        assert np.all(ct.mu >= 0) and ct.region.max() < ct.n_regions


def test_workload_sizes_match_their_recipe():
    cube = synth.cube_drop()
    assert cube.scene.X.shape[0] == 125 and cube.scene.tets.shape[0] == 320
    beam = synth.beam_incline()
    assert beam.scene.X.shape[0] == 4961 and beam.scene.tets.shape[0] == 20000
    assert beam.scene.contacts(beam.q0).n == 451
    ball = synth.sphere_press(cell=0.02)
    assert (ball.scene.X.shape[0], ball.scene.tets.shape[0], ball.scene.contacts(ball.q0).n) == (416, 2190, 119)
    blocks = synth.block_batch(64)
    assert len(blocks) == 64
    nt = [b.scene.tets.shape[0] for b in blocks]
    assert sum(nt) == 930875 and sum(b.scene.X.shape[0] for b in blocks) == 227449
    assert 1500 <= min(nt) and max(nt) <= 55000


def test_actuation_draws():
    a1, d1 = synth.random_actuation(100, seed=5)
    a2, d2 = synth.random_actuation(100, seed=5)
    assert a1.dtype == np.float32 and np.array_equal(a1, a2) and np.array_equal(d1, d2)
    assert np.allclose(np.linalg.norm(d1, axis=1), 1.0, atol=1e-12)
    a3, _ = synth.random_actuation(100, seed=6)
    assert not np.array_equal(a1, a3)


def test_cloth_grid_and_sphere_contacts():
    """The cloth recipe: an (n+1)^2 grid of 2 n^2 counter-clockwise triangles (alternating
    diagonals), above a sphere; each sphere contact's frame rows are orthonormal with the normal
    radial at the previous position, and n . x - d_n is the distance to the sphere there."""
    X, T = synth.tri_grid(4, 3, 0.4, 0.3)
    assert X.shape == (20, 3) and T.shape == (24, 3)
    e1, e2 = X[T[:, 1]] - X[T[:, 0]], X[T[:, 2]] - X[T[:, 0]]
    assert np.all(np.cross(e1, e2)[:, 2] > 0) and np.allclose(0.5 * np.cross(e1, e2)[:, 2].sum(), 0.12)
    pb = synth.cloth_drape()
    sc = pb.scene
    assert sc.X.shape[0] == 1024 and sc.tets.shape[0] == 1922 and sc.thickness > 0 and sc.bend > 0
    a, b = _arrays(pb), _arrays(synth.cloth_drape())
    for x, y in zip(a, b):
        assert np.asarray(x).tobytes() == np.asarray(y).tobytes()
    sph = synth.Sphere(np.array([0.1, -0.2, 0.0]), 0.3, mu=0.4)
    rng = np.random.default_rng(0)
    d = rng.normal(size=(50, 3))
    xp = sph.center + d / np.linalg.norm(d, axis=1)[:, None] * rng.uniform(0.29, 0.31, (50, 1))
    verts, frames, dn, mu, reg = sph.contacts(xp, 2e-3, np.arange(50), 0)
    assert len(verts) > 0 and np.all(mu == 0.4) and np.all(reg == 0)
    assert np.allclose(np.einsum("cij,ckj->cik", frames, frames), np.eye(3), atol=1e-12)
    assert np.all(np.linalg.det(frames) > 0)
    dist = np.linalg.norm(xp[verts] - sph.center, axis=1) - sph.radius
    assert np.all(dist < 2e-3)
    assert np.allclose(np.einsum("ci,ci->c", frames[:, 0], xp[verts]) - dn, dist, atol=1e-14)
    ct = synth.detect_contacts(xp, [], 2e-3, None, [sph])
    assert np.array_equal(ct.vertex, verts) and ct.n_regions == 1
