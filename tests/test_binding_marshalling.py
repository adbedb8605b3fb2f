"""The Python binding's argument marshalling (CPU only): a fake library stands in for the C entry
points and records the structs the binding fills in, so that pointers, counts, enum values, the
requested outputs and their shapes are checked without a device."""
import ctypes as C
import types

import pytest
import torch

from paper_2603_16478_gb300 import binding as B


class FakeLib:
    """Records the last call of each entry point; returns OK."""

    def __init__(self):
        self.calls = {}

    def ncpadj_options_default(self, opt_ref):
        o = opt_ref._obj
        o.eps, o.rtol, o.max_iters, o.gmres_restart = 1e-4, 1e-8, 2000, 64
        o.precision = o.precond = o.solver = o.memory = o.cap_precision = o.cap_block = 0
        o.precond = 3

    def ncpadj_adjoint_step(self, ctx, scene, cts, stt, sd, opt, gr, stats, stream):
        self.calls["adjoint"] = (cts._obj, stt._obj, sd._obj, opt._obj, gr._obj)
        stats._obj.iterations = 7
        return 0

    def ncpadj_forward_step(self, ctx, scene, cts, fin, opt, tol, max_newton, q, lam, stats, stream):
        self.calls["forward"] = (cts._obj, fin._obj, opt._obj, tol, max_newton)
        return 0

    def ncpadj_last_error(self):
        return b""


@pytest.fixture
def fake_scene():
    lib = FakeLib()
    sc = object.__new__(B.Scene)
    sc.lib, sc.handle, sc.n_verts, sc.n_tets = lib, C.c_void_p(1), 10, 12
    sc.ctx = types.SimpleNamespace(handle=C.c_void_p(2))
    return sc, lib


def _t(*shape, dt=torch.float64):
    return torch.zeros(*shape, dtype=dt)


def test_adjoint_marshalling_with_contacts_and_bindings(fake_scene):
    sc, lib = fake_scene
    ct = B.Contacts(_t(3, dt=torch.int32), _t(3, 3, 3), _t(3), _t(3), None, _t(3, dt=torch.int32), 4)
    bd = B.Bindings(None, _t(2, 3), _t(2) + 1e-4, tet=_t(2, dt=torch.int32), bary=_t(2, 4))
    q, qp, lam, dq = _t(10, 3), _t(10, 3), _t(3, 3), _t(10, 3)
    g, stats = B.adjoint_step(sc, ct, q, qp, lam, dq, None, eps=2e-4, rtol=1e-9, precision="mixed",
                              cap_precision="fp64", solver="bicgstab", precond="jacobi", restart=32, bindings=bd)
    cts, stt, sd, opt, gr = lib.calls["adjoint"]
    assert cts.n_contacts == 3 and cts.vertex == ct.vertex.data_ptr() and cts.n_regions == 4 and cts.d_f is None
    assert stt.q == q.data_ptr() and stt.lam == lam.data_ptr()
    b = stt.bindings.contents
    assert b.n_bindings == 2 and b.vertex is None and b.tet == bd.tet.data_ptr() and b.bary == bd.bary.data_ptr()
    assert sd.dL_dq == dq.data_ptr() and sd.dL_dv is None
    assert (opt.eps, opt.rtol, opt.gmres_restart) == (2e-4, 1e-9, 32)
    assert (opt.precision, opt.cap_precision, opt.solver, opt.precond) == (1, 0, 3, 1)
    shapes = {"dL_dq_prev": (10, 3), "dL_dE": (12,), "dL_dmu": (4,), "dL_dmu_contact": (3,),
              "dL_dbinding_target": (2, 3), "dL_dcompliance": (2,)}
    for k, shp in shapes.items():
        assert tuple(g[k].shape) == shp and getattr(gr, k) == g[k].data_ptr(), k
    assert gr.dL_dact is None and stats["iterations"] == 7


def test_adjoint_marshalling_without_optional_parts(fake_scene):
    sc, lib = fake_scene
    g, _ = B.adjoint_step(sc, None, _t(10, 3), _t(10, 3), _t(0, 3), _t(10, 3), None)
    cts, stt, sd, opt, gr = lib.calls["adjoint"]
    assert cts.n_contacts == 0 and cts.n_regions == 1 and not stt.bindings and stt.lam is None
    assert "dL_dbinding_target" not in g and gr.dL_dbinding_target is None and gr.dL_dcompliance is None
    assert (opt.precision, opt.solver, opt.precond) == (0, 0, 3)


def test_forward_marshalling_with_bindings_and_actuation(fake_scene):
    sc, lib = fake_scene
    bd = B.Bindings(_t(2, dt=torch.int32), _t(2, 3), _t(2) + 1e-4)
    act = torch.zeros(12, dtype=torch.float32)
    B.forward_step(sc, None, _t(10, 3), _t(10, 3), None, (0.0, 0.0, -9.0), eps=3e-4, newton_tol=1e-9, max_newton=77,
                   act=act, bindings=bd, cap_precision="mixed")
    cts, fin, opt, tol, mx = lib.calls["forward"]
    assert tuple(fin.gravity) == (0.0, 0.0, -9.0) and fin.act == act.data_ptr() and fin.f_ext is None
    b = fin.bindings.contents
    assert b.n_bindings == 2 and b.vertex == bd.vertex.data_ptr() and b.tet is None and b.bary is None
    assert (tol, mx, opt.eps, opt.cap_precision) == (1e-9, 77, 3e-4, 1)


def test_model_names_map_to_the_header_codes(fake_scene):
    sc, lib = fake_scene
    seen = {}

    def set_model(handle, ptr):
        seen["codes"] = list((C.c_int32 * sc.n_tets).from_address(ptr.value))
        return 0

    lib.ncpadj_scene_set_model = set_model
    sc.set_model("arap")
    assert seen["codes"] == [2] * 12
    sc.set_model(["neo_hookean", "corotational", 2] * 4)
    assert seen["codes"] == [0, 1, 2] * 4
    with pytest.raises(ValueError):
        sc.set_model(["arap"] * 3)


def test_scene_descriptors_single_and_batch():
    """Scene construction passes one descriptor (or one per mesh of a batch) with host copies of
    the arrays, E and nu broadcast per tet, and numbers the batch's meshes one after another."""
    import numpy as np
    lib = FakeLib()
    seen = {}

    def create(ctx, desc_ref, out_ref):
        d = desc_ref._obj
        seen["single"] = (d.n_verts, d.n_tets, d.density, d.h,
                          list((C.c_double * d.n_tets).from_address(d.E)), list((C.c_int32 * 4).from_address(d.tets)))
        out_ref._obj.value = 11
        return 0

    def create_batch(ctx, n, descs, out_ref):
        seen["batch"] = [(descs[i].n_verts, descs[i].n_tets, descs[i].density) for i in range(n)]
        seen["nu0"] = list((C.c_double * descs[0].n_tets).from_address(descs[0].nu))
        out_ref._obj.value = 12
        return 0

    lib.ncpadj_scene_create = create
    lib.ncpadj_scene_create_batch = create_batch
    ctx = types.SimpleNamespace(lib=lib, handle=C.c_void_p(2))
    X = np.zeros((5, 3))
    T = np.array([[0, 1, 2, 3], [1, 2, 3, 4]])
    sc = B.Scene(ctx, X, T, 1e5, 0.4, 1000.0, 0.01)
    assert seen["single"] == (5, 2, 1000.0, 0.01, [1e5, 1e5], [0, 1, 2, 3])
    assert (sc.n_verts, sc.n_tets, sc.handle.value) == (5, 2, 11)
    sb = B.Scene.batch(ctx, [(X, T, 1e5, 0.4, 1000.0), (np.zeros((4, 3)), T[:1], [2e5], [0.3], 900.0)], 0.01)
    assert seen["batch"] == [(5, 2, 1000.0), (4, 1, 900.0)] and seen["nu0"] == [0.4, 0.4]
    assert sb.vertex_offsets == [0, 5, 9] and sb.tet_offsets == [0, 2, 3] and (sb.n_verts, sb.n_tets) == (9, 3)
    sb.handle = sc.handle = C.c_void_p()  # nothing to destroy in the fake
