"""ctypes binding of ``include/ncpadj.h`` (argument marshalling only).

Tensors are passed by pointer: CUDA tensors with ``memory="device"``, CPU tensors (pinned
memory recommended) with ``memory="host"``.  float64 everywhere except int32 indices.
"""
from __future__ import annotations

import ctypes as C
import os
from dataclasses import dataclass
from typing import Optional

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
_LIB = None

STATUS = ["OK", "INVALID_ARG", "CUDA", "OOM", "INVERTED_ELEMENT", "NOT_CONVERGED", "NONFINITE", "TIMEOUT",
          "NOT_FACTORED", "UNSUPPORTED", "CONTACT_DOMAIN"]
PRECOND = {"none": 0, "jacobi": 1, "elastic": 2, "woodbury": 3}
SOLVER = {"auto": 0, "cg": 1, "gmres": 2, "bicgstab": 3, "semi_implicit": 4}
PRECISION = {"fp64": 0, "mixed": 1, "tf32x3": 2, "refined": 3}  # "refined": capacitance precision only
MEMORY = {"device": 0, "host": 1}
MODEL = {"neo_hookean": 0, "corotational": 1, "arap": 2}


def library_path() -> str:
    return os.path.join(_HERE, "libncpadj.so")


class NcpadjError(RuntimeError):
    def __init__(self, status: int, message: str, stats=None, grads=None):
        super().__init__(f"ncpadj {status_name(status)}: {message}")
        self.status = status
        self.stats = stats
        self.grads = grads


def status_name(s: int) -> str:
    return STATUS[s] if 0 <= s < len(STATUS) else f"status {s}"


class _SceneDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("rest_pos", C.c_void_p), ("tets", C.c_void_p),
                ("E", C.c_void_p), ("nu", C.c_void_p), ("density", C.c_double), ("h", C.c_double)]


class _ShellDesc(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tris", C.c_int32), ("rest_pos", C.c_void_p), ("tris", C.c_void_p),
                ("E", C.c_void_p), ("nu", C.c_void_p), ("density", C.c_double), ("h", C.c_double),
                ("thickness", C.c_double), ("bend", C.c_double)]


class _SceneInfo(C.Structure):
    _fields_ = [("n_verts", C.c_int32), ("n_tets", C.c_int32), ("n_blocks", C.c_int32), ("nnz_L", C.c_int64),
                ("nnz_Linv", C.c_int64), ("ms_factor", C.c_double), ("n_scenes", C.c_int32),
                ("element_verts", C.c_int32), ("n_hinges", C.c_int32)]


class _Contacts(C.Structure):
    _fields_ = [("n_contacts", C.c_int32), ("vertex", C.c_void_p), ("frame", C.c_void_p), ("d_n", C.c_void_p),
                ("d_f", C.c_void_p), ("mu", C.c_void_p), ("region", C.c_void_p), ("n_regions", C.c_int32)]


class _Bindings(C.Structure):
    _fields_ = [("n_bindings", C.c_int32), ("vertex", C.c_void_p), ("target", C.c_void_p),
                ("compliance", C.c_void_p), ("tet", C.c_void_p), ("bary", C.c_void_p)]


class _State(C.Structure):
    _fields_ = [("q", C.c_void_p), ("q_prev", C.c_void_p), ("lam", C.c_void_p),
                ("bindings", C.POINTER(_Bindings))]


class _Seed(C.Structure):
    _fields_ = [("dL_dq", C.c_void_p), ("dL_dv", C.c_void_p)]


class _Grads(C.Structure):
    _fields_ = [("dL_dq_prev", C.c_void_p), ("dL_dv_prev", C.c_void_p), ("dL_dfext", C.c_void_p),
                ("dL_dE", C.c_void_p), ("dL_dnu", C.c_void_p), ("dL_dmu", C.c_void_p),
                ("dL_dmu_contact", C.c_void_p), ("z", C.c_void_p), ("dL_dact", C.c_void_p),
                ("dL_dbinding_target", C.c_void_p), ("dL_dcompliance", C.c_void_p), ("dL_dbend", C.c_void_p)]


class _Options(C.Structure):
    _fields_ = [("eps", C.c_double), ("rtol", C.c_double), ("max_iters", C.c_int32), ("gmres_restart", C.c_int32),
                ("precision", C.c_int32), ("precond", C.c_int32), ("solver", C.c_int32), ("memory", C.c_int32),
                ("cap_precision", C.c_int32), ("cap_block", C.c_int32), ("cap_drop", C.c_double)]


class _Stats(C.Structure):
    _fields_ = [("iterations", C.c_int32), ("solver_used", C.c_int32), ("n_contacts", C.c_int32),
                ("capacitance_dim", C.c_int32), ("rel_residual", C.c_double), ("ms_total", C.c_float),
                ("ms_assemble", C.c_float), ("ms_setup", C.c_float), ("ms_krylov", C.c_float),
                ("ms_contract", C.c_float), ("ms_cap_inverse", C.c_float), ("kernel_launches", C.c_int64),
                ("capacitance_blocks", C.c_int32), ("inner_iterations", C.c_int32)]

    def to_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


class _ForwardInput(C.Structure):
    _fields_ = [("q_prev", C.c_void_p), ("v_prev", C.c_void_p), ("f_ext", C.c_void_p), ("gravity", C.c_double * 3),
                ("act", C.c_void_p), ("bindings", C.POINTER(_Bindings))]


class _ForwardStats(C.Structure):
    _fields_ = [("newton_iters", C.c_int32), ("krylov_iters", C.c_int32), ("residual", C.c_double),
                ("ms_total", C.c_float)]

    def to_dict(self):
        return {f: getattr(self, f) for f, _ in self._fields_}


EXPORTS = ["ncpadj_version", "ncpadj_status_string", "ncpadj_last_error", "ncpadj_ctx_create", "ncpadj_ctx_destroy",
           "ncpadj_scene_create", "ncpadj_scene_create_batch", "ncpadj_scene_destroy", "ncpadj_scene_get_info",
           "ncpadj_scene_refactor", "ncpadj_scene_get_material", "ncpadj_scene_create_shells",
           "ncpadj_scene_set_bending", "ncpadj_scene_get_bending",
           "ncpadj_options_default", "ncpadj_adjoint_step", "ncpadj_adjoint_batch", "ncpadj_forward_step",
           "ncpadj_elastic_solve", "ncpadj_elastic_solve_noalloc", "ncpadj_elastic_solve_mixed", "ncpadj_dense_inverse",
           "ncpadj_dense_gemm",
           "ncpadj_scene_set_fibres", "ncpadj_scene_set_model", "ncpadj_scene_set_chunk"]


def load_library(path: Optional[str] = None):
    """Load libncpadj.so (raises if it is missing: there is no fallback)."""
    global _LIB
    if _LIB is not None and path is None:
        return _LIB
    p = path or library_path()
    if not os.path.exists(p):
        raise RuntimeError(f"{p} is missing: build the CUDA library first (python -c 'import __graft_entry__ as g; "
                           "g.build()')")
    lib = C.CDLL(p)
    lib.ncpadj_version.restype = C.c_char_p
    lib.ncpadj_status_string.restype = C.c_char_p
    lib.ncpadj_status_string.argtypes = [C.c_int]
    lib.ncpadj_last_error.restype = C.c_char_p
    lib.ncpadj_ctx_create.argtypes = [C.c_int, C.POINTER(C.c_void_p)]
    lib.ncpadj_ctx_destroy.argtypes = [C.c_void_p]
    lib.ncpadj_scene_create.argtypes = [C.c_void_p, C.POINTER(_SceneDesc), C.POINTER(C.c_void_p)]
    lib.ncpadj_scene_destroy.argtypes = [C.c_void_p]
    lib.ncpadj_scene_create_batch.argtypes = [C.c_void_p, C.c_int32, C.POINTER(_SceneDesc), C.POINTER(C.c_void_p)]
    lib.ncpadj_scene_get_info.argtypes = [C.c_void_p, C.POINTER(_SceneInfo)]
    lib.ncpadj_scene_create_shells.argtypes = [C.c_void_p, C.c_int32, C.POINTER(_ShellDesc), C.POINTER(C.c_void_p)]
    lib.ncpadj_scene_set_bending.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ncpadj_scene_get_bending.argtypes = [C.c_void_p, C.c_void_p]
    lib.ncpadj_scene_refactor.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ncpadj_scene_get_material.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ncpadj_options_default.argtypes = [C.POINTER(_Options)]
    lib.ncpadj_adjoint_step.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(_Contacts), C.POINTER(_State),
                                        C.POINTER(_Seed), C.POINTER(_Options), C.POINTER(_Grads), C.POINTER(_Stats),
                                        C.c_void_p]
    lib.ncpadj_adjoint_batch.argtypes = [C.c_void_p, C.c_void_p, C.c_int32, C.POINTER(_Contacts), C.POINTER(_State),
                                         C.POINTER(_Seed), C.POINTER(_Options), C.POINTER(_Grads),
                                         C.POINTER(_Stats), C.c_void_p]
    lib.ncpadj_forward_step.argtypes = [C.c_void_p, C.c_void_p, C.POINTER(_Contacts), C.POINTER(_ForwardInput),
                                        C.POINTER(_Options), C.c_double, C.c_int32, C.c_void_p, C.c_void_p,
                                        C.POINTER(_ForwardStats), C.c_void_p]
    lib.ncpadj_elastic_solve.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ncpadj_elastic_solve_noalloc.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ncpadj_elastic_solve_mixed.argtypes = [C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p, C.c_void_p]
    lib.ncpadj_scene_set_fibres.argtypes = [C.c_void_p, C.c_void_p]
    lib.ncpadj_scene_set_model.argtypes = [C.c_void_p, C.c_void_p]
    lib.ncpadj_dense_inverse.argtypes = [C.c_void_p, C.c_int32, C.c_void_p, C.c_void_p, C.c_int32, C.c_void_p]
    lib.ncpadj_scene_set_chunk.argtypes = [C.c_void_p, C.c_int32]
    lib.ncpadj_dense_gemm.argtypes = [C.c_void_p, C.c_int32, C.c_int32, C.c_int32, C.c_float, C.c_void_p, C.c_int64,
                                      C.c_void_p, C.c_int64, C.c_float, C.c_void_p, C.c_int64, C.c_int32, C.c_void_p]
    if path is None:
        _LIB = lib
    return lib


def _check(lib, st):
    if st != 0:
        raise NcpadjError(st, lib.ncpadj_last_error().decode())


def _ptr(t: Optional[torch.Tensor]):
    return None if t is None else C.c_void_p(t.data_ptr())


class Context:
    def __init__(self, device: int = 0):
        self.lib = load_library()
        h = C.c_void_p()
        _check(self.lib, self.lib.ncpadj_ctx_create(device, C.byref(h)))
        self.handle = h
        self.device = device

    def close(self):
        if self.handle:
            self.lib.ncpadj_ctx_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


class Scene:
    """Mesh + material + step size; builds the elastic factor on construction (host arrays).

    ``Scene.batch(ctx, meshes, h)`` builds a batch: the disjoint union of several meshes, each
    ``(X, tets, E, nu, density)``, numbered one after the other (``vertex_offsets``).
    ``Scene.shells(ctx, meshes, h)`` builds one or more triangle meshes (shells), each
    ``(X, tris, E, nu, density, thickness, bend)``; their elements take the place of the tets
    (``n_tets`` counts triangles)."""

    chunk = 256  # chunk length of the A^{-1} product (set_chunk)

    def __init__(self, ctx: Context, X, tets, E, nu, density: float, h: float, _batch=None, _shells=None):
        self.ctx = ctx
        self.lib = ctx.lib
        if _shells is not None:
            meshes = _shells
        else:
            meshes = [m + (0.0, 0.0) for m in (_batch if _batch is not None else [(X, tets, E, nu, density)])]
        self._keep = []
        descs = (_ShellDesc if _shells is not None else _SceneDesc) * len(meshes)
        descs = descs()
        offs = [0]
        toffs = [0]
        for i, (Xi, Ti, Ei, nui, rho, tau, kb) in enumerate(meshes):
            Xt = torch.as_tensor(Xi, dtype=torch.float64).contiguous().cpu()
            Tt = torch.as_tensor(Ti, dtype=torch.int32).contiguous().cpu()
            nt = Tt.shape[0]
            Et = torch.as_tensor(Ei, dtype=torch.float64).expand(nt).contiguous().cpu()
            nut = torch.as_tensor(nui, dtype=torch.float64).expand(nt).contiguous().cpu()
            self._keep += [Xt, Tt, Et, nut]
            args = (Xt.shape[0], nt, Xt.data_ptr(), Tt.data_ptr(), Et.data_ptr(), nut.data_ptr(), float(rho), float(h))
            descs[i] = _ShellDesc(*args, float(tau), float(kb)) if _shells is not None else _SceneDesc(*args)
            offs.append(offs[-1] + Xt.shape[0])
            toffs.append(toffs[-1] + nt)
        hnd = C.c_void_p()
        if _shells is not None:
            _check(self.lib, self.lib.ncpadj_scene_create_shells(ctx.handle, len(meshes), descs, C.byref(hnd)))
        elif _batch is None:
            _check(self.lib, self.lib.ncpadj_scene_create(ctx.handle, C.byref(descs[0]), C.byref(hnd)))
        else:
            _check(self.lib, self.lib.ncpadj_scene_create_batch(ctx.handle, len(meshes), descs, C.byref(hnd)))
        self.handle = hnd
        self.vertex_offsets = offs
        self.tet_offsets = toffs
        self.n_verts = offs[-1]
        self.n_tets = toffs[-1]
        self.h = float(h)

    @classmethod
    def batch(cls, ctx: Context, meshes, h: float) -> "Scene":
        return cls(ctx, None, None, None, None, None, h, _batch=list(meshes))

    @classmethod
    def shells(cls, ctx: Context, meshes, h: float) -> "Scene":
        return cls(ctx, None, None, None, None, None, h, _shells=list(meshes))

    @property
    def n_scenes(self) -> int:
        return len(self.vertex_offsets) - 1

    def set_bending(self, bend, stream=None) -> None:
        """New bending stiffness of each shell mesh (scalar or [n_scenes]); rebuilds the elastic factor."""
        b = torch.as_tensor(bend, dtype=torch.float64).expand(self.n_scenes).contiguous().cpu()
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(self.ctx.device).cuda_stream
        _check(self.lib, self.lib.ncpadj_scene_set_bending(self.handle, C.c_void_p(b.data_ptr()),
                                                           C.c_void_p(stream or 0)))

    def bending(self):
        """The bending stiffness of each mesh (CPU float64 [n_scenes]; zeros for tet scenes)."""
        b = torch.empty(self.n_scenes, dtype=torch.float64)
        _check(self.lib, self.lib.ncpadj_scene_get_bending(self.handle, C.c_void_p(b.data_ptr())))
        return b

    def set_fibres(self, fibre) -> None:
        """Unit fibre directions [n_tets, 3] of the per-tet actuation (host array)."""
        f = torch.as_tensor(fibre, dtype=torch.float64).reshape(-1, 3).contiguous().cpu()
        if f.shape[0] != self.n_tets:
            raise ValueError(f"expected {self.n_tets} fibres, got {f.shape[0]}")
        self._fibre = f
        _check(self.lib, self.lib.ncpadj_scene_set_fibres(self.handle, C.c_void_p(f.data_ptr())))

    def set_chunk(self, entries: int) -> None:
        """Chunk length (128, 256 or 512 nonzeros per warp) of the A^{-1} product's kernels; a launch
        shape the autotuner picks by timing."""
        _check(self.lib, self.lib.ncpadj_scene_set_chunk(self.handle, int(entries)))
        self.chunk = int(entries)

    def set_model(self, model) -> None:
        """Constitutive model of every tet (App. B.2): one of "neo_hookean", "corotational", "arap",
        or a per-tet sequence of those names or of their codes (MODEL)."""
        if isinstance(model, str):
            codes = [MODEL[model]] * self.n_tets
        else:
            codes = [MODEL[m] if isinstance(m, str) else int(m) for m in model]
        if len(codes) != self.n_tets:
            raise ValueError(f"expected {self.n_tets} models, got {len(codes)}")
        m = torch.tensor(codes, dtype=torch.int32)
        _check(self.lib, self.lib.ncpadj_scene_set_model(self.handle, C.c_void_p(m.data_ptr())))

    def refactor(self, E, nu, stream=None) -> None:
        """New per-tet (or scalar) Young's modulus and Poisson ratio: the material-dependent arrays and
        the elastic factor are rebuilt (host-side factorisation; synchronous)."""
        Et = torch.as_tensor(E, dtype=torch.float64).expand(self.n_tets).contiguous().cpu()
        nut = torch.as_tensor(nu, dtype=torch.float64).expand(self.n_tets).contiguous().cpu()
        if stream is None and torch.cuda.is_available():
            stream = torch.cuda.current_stream(self.ctx.device).cuda_stream
        _check(self.lib, self.lib.ncpadj_scene_refactor(self.handle, C.c_void_p(Et.data_ptr()),
                                                        C.c_void_p(nut.data_ptr()), C.c_void_p(stream or 0)))

    def material(self):
        """(E, nu): the scene's current per-tet material (CPU float64 tensors [n_tets])."""
        E = torch.empty(self.n_tets, dtype=torch.float64)
        nu = torch.empty(self.n_tets, dtype=torch.float64)
        _check(self.lib, self.lib.ncpadj_scene_get_material(self.handle, C.c_void_p(E.data_ptr()),
                                                            C.c_void_p(nu.data_ptr())))
        return E, nu

    def info(self) -> dict:
        inf = _SceneInfo()
        _check(self.lib, self.lib.ncpadj_scene_get_info(self.handle, C.byref(inf)))
        return {f: getattr(inf, f) for f, _ in inf._fields_}

    def close(self):
        if self.handle:
            self.lib.ncpadj_scene_destroy(self.handle)
            self.handle = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass


@dataclass
class Contacts:
    """Vertex-plane contacts (tensors on the device the call uses)."""
    vertex: torch.Tensor               # int32 [n_c]
    frame: torch.Tensor                # float64 [n_c, 3, 3] rows n, t1, t2
    d_n: torch.Tensor                  # float64 [n_c]
    mu: torch.Tensor                   # float64 [n_c]
    d_f: Optional[torch.Tensor] = None       # float64 [n_c, 2]
    region: Optional[torch.Tensor] = None    # int32 [n_c]
    n_regions: int = 1

    @property
    def n(self):
        return int(self.vertex.shape[0])

    def to(self, device):
        f = lambda t: None if t is None else t.to(device)  # noqa: E731
        return Contacts(f(self.vertex), f(self.frame), f(self.d_n), f(self.mu), f(self.d_f), f(self.region),
                        self.n_regions)


@dataclass
class Bindings:
    """Bilateral bindings (Eq. binding): a vertex, or with ``tet`` and ``bary`` the point
    sum_a bary[b, a] x_a of the vertices of tet[b], held near target[b] by a spring of compliance
    E_b (tensors on the device the call uses).  ``vertex`` may be None for points inside tets."""
    vertex: Optional[torch.Tensor]     # int32 [n_b]
    target: torch.Tensor               # float64 [n_b, 3]
    compliance: torch.Tensor           # float64 [n_b], > 0
    tet: Optional[torch.Tensor] = None   # int32 [n_b]
    bary: Optional[torch.Tensor] = None  # float64 [n_b, 4]

    @property
    def n(self):
        return int(self.compliance.shape[0])


def _bindings_ref(bindings: Optional[Bindings]):
    """(pointer for the call, the struct it points to: keep it alive for the call)."""
    if bindings is None or bindings.n == 0:
        return None, None
    b = _Bindings(bindings.n, _ptr(bindings.vertex), _ptr(bindings.target), _ptr(bindings.compliance),
                  _ptr(bindings.tet), _ptr(bindings.bary))
    return C.pointer(b), b


def adjoint_step(scene: Scene, contacts: Optional[Contacts], q, q_prev, lam, dL_dq, dL_dv=None, *, eps=1e-4,
                 rtol=1e-8, max_iters=2000, restart=64, precision="fp64", cap_precision="fp64", precond="woodbury",
                 solver="auto", cap_block=0, cap_drop=1e-2,
                 memory="device", outputs: Optional[dict] = None, stream=None, want=("dL_dq_prev", "dL_dv_prev",
                 "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu", "dL_dmu_contact", "z"), bindings: Optional[Bindings] = None):
    """One adjoint step through the C-ABI.  Returns (grads dict of tensors, stats dict).

    ``outputs`` may hold preallocated output tensors by name; otherwise they are allocated on
    q's device (pinned CPU memory with memory="host").  With ``bindings`` (the ones the forward
    step used) the outputs also hold dL_dbinding_target [n_b, 3] and dL_dcompliance [n_b].
    """
    lib = scene.lib
    nc = contacts.n if contacts is not None else 0
    nb = bindings.n if bindings is not None else 0
    nv, nt = scene.n_verts, scene.n_tets
    nreg = contacts.n_regions if contacts is not None else 1
    dev = q.device
    outputs = dict(outputs or {})
    if nb:
        want = tuple(want) + tuple(k for k in ("dL_dbinding_target", "dL_dcompliance") if k not in want)
    shapes = {"dL_dq_prev": (nv, 3), "dL_dv_prev": (nv, 3), "dL_dfext": (nv, 3), "z": (nv, 3), "dL_dE": (nt,),
              "dL_dnu": (nt,), "dL_dmu": (nreg,), "dL_dmu_contact": (max(nc, 0),), "dL_dact": (nt,),
              "dL_dbinding_target": (nb, 3), "dL_dcompliance": (nb,)}
    if "dL_dbend" in want:
        shapes["dL_dbend"] = (scene.n_scenes,)
    for k in want:
        if k not in outputs:
            dt = torch.float32 if k == "dL_dact" else torch.float64
            if memory == "host":
                outputs[k] = torch.empty(shapes[k], dtype=dt, pin_memory=torch.cuda.is_available())
            else:
                outputs[k] = torch.empty(shapes[k], dtype=dt, device=dev)
    cts = _Contacts(0, None, None, None, None, None, None, 1)
    if nc:
        cts = _Contacts(nc, _ptr(contacts.vertex), _ptr(contacts.frame), _ptr(contacts.d_n), _ptr(contacts.d_f),
                        _ptr(contacts.mu), _ptr(contacts.region), int(contacts.n_regions))
    bptr, _bkeep = _bindings_ref(bindings)
    stt = _State(_ptr(q), _ptr(q_prev), _ptr(lam) if nc else None, bptr)
    sd = _Seed(_ptr(dL_dq), _ptr(dL_dv))
    gr = _Grads(*[_ptr(outputs.get(k)) for k in _GRAD_FIELDS])
    opt = _Options()
    lib.ncpadj_options_default(C.byref(opt))
    opt.eps, opt.rtol, opt.max_iters, opt.gmres_restart = float(eps), float(rtol), int(max_iters), int(restart)
    opt.precision = PRECISION[precision]
    opt.cap_precision = PRECISION[cap_precision]
    opt.cap_block = int(cap_block)
    opt.cap_drop = float(cap_drop)
    opt.precond = PRECOND[precond]
    opt.solver = SOLVER[solver]
    opt.memory = MEMORY[memory]
    stats = _Stats()
    if stream is None and dev.type == "cuda":
        stream = torch.cuda.current_stream(dev).cuda_stream
    st = lib.ncpadj_adjoint_step(scene.ctx.handle, scene.handle, C.byref(cts), C.byref(stt), C.byref(sd),
                                 C.byref(opt), C.byref(gr), C.byref(stats), C.c_void_p(stream or 0))
    if st != 0:
        raise NcpadjError(st, lib.ncpadj_last_error().decode(), stats.to_dict(), outputs)
    return outputs, stats.to_dict()


_GRAD_FIELDS = ("dL_dq_prev", "dL_dv_prev", "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu", "dL_dmu_contact", "z", "dL_dact",
                "dL_dbinding_target", "dL_dcompliance", "dL_dbend")


def _options(lib, eps, rtol, max_iters, restart, precision, cap_precision, precond, solver, memory, cap_block,
             cap_drop=1e-2):
    opt = _Options()
    lib.ncpadj_options_default(C.byref(opt))
    opt.eps, opt.rtol, opt.max_iters, opt.gmres_restart = float(eps), float(rtol), int(max_iters), int(restart)
    opt.precision = PRECISION[precision]
    opt.cap_precision = PRECISION[cap_precision]
    opt.cap_block = int(cap_block)
    opt.cap_drop = float(cap_drop)
    opt.precond = PRECOND[precond]
    opt.solver = SOLVER[solver]
    opt.memory = MEMORY[memory]
    return opt


class BatchCall:
    """A prepared ``ncpadj_adjoint_batch`` call: the per-mesh argument structs are built once, so
    that repeated calls (same tensors, new values) cost one library call each.

    ``contacts``, ``q``, ``q_prev``, ``lam``, ``dL_dq`` (and ``dL_dv``, or None) are lists with one
    entry per mesh of a batch scene (``Scene.batch``), in the mesh's own numbering; ``contacts[s]``
    may be None (``lam[s]`` is then ignored).  ``outputs`` may give the per-mesh output tensors
    (list of dicts by name); missing ones are allocated on the inputs' device (pinned CPU memory
    with memory="host").  ``run()`` returns the per-mesh stats dicts; the outputs are in
    ``self.outputs``."""

    def __init__(self, scene: Scene, contacts, q, q_prev, lam, dL_dq, dL_dv=None, *, eps=1e-4, rtol=1e-8,
                 max_iters=2000, restart=64, precision="fp64", cap_precision="fp64", precond="woodbury",
                 cap_block=0, cap_drop=1e-2, memory="device", outputs=None,
                 want=("dL_dq_prev", "dL_dv_prev", "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu", "dL_dmu_contact", "z")):
        lib = self.lib = scene.lib
        self.scene = scene
        ns = self.ns = len(scene.vertex_offsets) - 1
        for name, lst in (("contacts", contacts), ("q", q), ("q_prev", q_prev), ("lam", lam), ("dL_dq", dL_dq)):
            if len(lst) != ns:
                raise ValueError(f"{name}: expected {ns} entries (one per mesh), got {len(lst)}")
        if dL_dv is not None and len(dL_dv) != ns:
            raise ValueError(f"dL_dv: expected {ns} entries, got {len(dL_dv)}")
        self.device = q[0].device
        self._keep = (contacts, q, q_prev, lam, dL_dq, dL_dv)
        self.cts, self.stt = (_Contacts * ns)(), (_State * ns)()
        self.sds, self.grs = (_Seed * ns)(), (_Grads * ns)()
        self.outputs = []
        for s in range(ns):
            nv = scene.vertex_offsets[s + 1] - scene.vertex_offsets[s]
            nt = scene.tet_offsets[s + 1] - scene.tet_offsets[s]
            ct = contacts[s]
            nc = ct.n if ct is not None else 0
            nreg = ct.n_regions if ct is not None else 1
            shapes = {"dL_dq_prev": (nv, 3), "dL_dv_prev": (nv, 3), "dL_dfext": (nv, 3), "z": (nv, 3), "dL_dE": (nt,),
                      "dL_dnu": (nt,), "dL_dmu": (nreg,), "dL_dmu_contact": (nc,), "dL_dact": (nt,),
                      "dL_dbend": (1,)}
            o = dict(outputs[s]) if outputs is not None else {}
            for k in want:
                if k in o:
                    continue
                dt = torch.float32 if k == "dL_dact" else torch.float64
                if memory == "host":
                    o[k] = torch.empty(shapes[k], dtype=dt, pin_memory=torch.cuda.is_available())
                else:
                    o[k] = torch.empty(shapes[k], dtype=dt, device=self.device)
            self.outputs.append(o)
            self.cts[s] = _contacts_struct(ct)
            self.stt[s] = _State(_ptr(q[s]), _ptr(q_prev[s]), _ptr(lam[s]) if nc else None, None)
            self.sds[s] = _Seed(_ptr(dL_dq[s]), _ptr(dL_dv[s]) if dL_dv is not None else None)
            self.grs[s] = _Grads(*[_ptr(o.get(k)) for k in _GRAD_FIELDS])
        self.opt = _options(lib, eps, rtol, max_iters, restart, precision, cap_precision, precond, "gmres", memory,
                            cap_block, cap_drop)
        self.stats = (_Stats * ns)()

    def run(self, stream=None):
        if stream is None and self.device.type == "cuda":
            stream = torch.cuda.current_stream(self.device).cuda_stream
        st = self.lib.ncpadj_adjoint_batch(self.scene.ctx.handle, self.scene.handle, self.ns, self.cts, self.stt,
                                           self.sds, C.byref(self.opt), self.grs, self.stats, C.c_void_p(stream or 0))
        sl = [self.stats[s].to_dict() for s in range(self.ns)]
        if st != 0:
            raise NcpadjError(st, self.lib.ncpadj_last_error().decode(), sl, self.outputs)
        return sl


def adjoint_batch(scene: Scene, contacts, q, q_prev, lam, dL_dq, dL_dv=None, *, stream=None, **kw):
    """One adjoint step of every mesh of a batch scene (``Scene.batch``) through
    ``ncpadj_adjoint_batch``: every mesh runs its own GMRES, sharing the launches.  Arguments as
    ``BatchCall``; returns (list of per-mesh output dicts, list of per-mesh stats dicts)."""
    call = BatchCall(scene, contacts, q, q_prev, lam, dL_dq, dL_dv, **kw)
    return call.outputs, call.run(stream)


def _contacts_struct(contacts):
    if contacts is None or contacts.n == 0:
        return _Contacts(0, None, None, None, None, None, None, 1)
    return _Contacts(contacts.n, _ptr(contacts.vertex), _ptr(contacts.frame), _ptr(contacts.d_n), _ptr(contacts.d_f),
                     _ptr(contacts.mu), _ptr(contacts.region), int(contacts.n_regions))


def forward_step(scene: Scene, contacts: Optional[Contacts], q_prev, v_prev=None, f_ext=None,
                 gravity=(0.0, 0.0, -9.81), *, eps=1e-4, newton_tol=1e-10, max_newton=60, precond="woodbury",
                 rtol=1e-10, max_iters=2000, restart=64, stream=None, act=None, cap_precision="fp64",
                 bindings: Optional[Bindings] = None):
    """One forward step on the GPU (device tensors).  ``act``: float32 [n_tets] activations (the
    scene needs fibres, ``Scene.set_fibres``); ``bindings``: bilateral bindings of the step.
    Returns (q, lambda [n_c, 3], stats)."""
    lib = scene.lib
    nc = contacts.n if contacts is not None else 0
    dev = q_prev.device
    q = torch.empty_like(q_prev)
    lam = torch.empty((max(nc, 1), 3), dtype=torch.float64, device=dev)
    bptr, _bkeep = _bindings_ref(bindings)
    fin = _ForwardInput(_ptr(q_prev), _ptr(v_prev), _ptr(f_ext), (C.c_double * 3)(*[float(g) for g in gravity]),
                        _ptr(act), bptr)
    opt = _Options()
    lib.ncpadj_options_default(C.byref(opt))
    opt.eps, opt.rtol, opt.max_iters, opt.gmres_restart = float(eps), float(rtol), int(max_iters), int(restart)
    opt.precond = PRECOND[precond]
    opt.cap_precision = PRECISION[cap_precision]  # "mixed": FP32 capacitance (it only preconditions)
    stats = _ForwardStats()
    if stream is None and dev.type == "cuda":
        stream = torch.cuda.current_stream(dev).cuda_stream
    cts = _contacts_struct(contacts)
    st = lib.ncpadj_forward_step(scene.ctx.handle, scene.handle, C.byref(cts), C.byref(fin), C.byref(opt),
                                 float(newton_tol), int(max_newton), _ptr(q), _ptr(lam), C.byref(stats),
                                 C.c_void_p(stream or 0))
    if st != 0:
        err = NcpadjError(st, lib.ncpadj_last_error().decode(), stats.to_dict())
        if status_name(st) == "NOT_CONVERGED":
            err.state = (q, lam[:nc])  # the last iterate (its residual is in err.stats)
        raise err
    return q, lam[:nc], stats.to_dict()


def elastic_solve(scene: Scene, x: torch.Tensor, y: Optional[torch.Tensor] = None, stream=None,
                  precision: str = "fp64"):
    """y = A^{-1} x with the scene's elastic factor (device tensors [n_verts, 3]); precision "mixed"
    uses the FP32 values and intermediates of the mixed preconditioner."""
    lib = scene.lib
    y = torch.empty_like(x) if y is None else y
    if stream is None:
        stream = torch.cuda.current_stream(x.device).cuda_stream
    fn = lib.ncpadj_elastic_solve_mixed if precision == "mixed" else lib.ncpadj_elastic_solve
    _check(lib, fn(scene.ctx.handle, scene.handle, _ptr(x), _ptr(y), C.c_void_p(stream)))
    return y


def elastic_solve_noalloc(scene: Scene, x: torch.Tensor, y: torch.Tensor, stream=None):
    """y = A^{-1} x without device allocation in the call (y preallocated by the caller; scenes
    of at most 262,144 vertices; concurrent calls race on the library's static scratch)."""
    lib = scene.lib
    for name, t in (("x", x), ("y", y)):
        if (t.dtype != torch.float64 or not t.is_cuda or t.device.index != scene.ctx.device or not t.is_contiguous()
                or tuple(t.shape) != (scene.n_verts, 3)):
            raise ValueError(f"{name}: expected a contiguous float64 CUDA tensor of shape ({scene.n_verts}, 3) on "
                             f"device {scene.ctx.device}")
    if stream is None:
        stream = torch.cuda.current_stream(x.device).cuda_stream
    _check(lib, lib.ncpadj_elastic_solve_noalloc(scene.ctx.handle, scene.handle, _ptr(x), _ptr(y),
                                                 C.c_void_p(stream)))
    return y


def dense_gemm(ctx: Context, A: torch.Tensor, B: torch.Tensor, Cout: Optional[torch.Tensor] = None,
               alpha: float = 1.0, beta: float = 0.0, split: bool = True, stream=None) -> torch.Tensor:
    """C = alpha A B + beta C on the tensor cores (ncpadj_dense_gemm): FP32 CUDA matrices with unit
    column stride (row strides are the leading dimensions); split=True is 3xTF32 (about FP32
    accuracy), False plain TF32."""
    lib = ctx.lib
    for name, t in (("A", A), ("B", B)) + ((("C", Cout),) if Cout is not None else ()):
        if t.dim() != 2 or t.dtype != torch.float32 or not t.is_cuda or t.stride(1) != 1:
            raise ValueError(f"{name}: expected a 2-D float32 CUDA matrix with unit column stride")
    M, K = A.shape
    if B.shape[0] != K:
        raise ValueError(f"inner dimensions differ: {K} and {B.shape[0]}")
    N = B.shape[1]
    if Cout is None:
        Cout = torch.zeros((M, N), dtype=torch.float32, device=A.device)
    elif tuple(Cout.shape) != (M, N):
        raise ValueError(f"C: expected shape {(M, N)}, got {tuple(Cout.shape)}")
    if stream is None:
        stream = torch.cuda.current_stream(A.device).cuda_stream
    _check(lib, lib.ncpadj_dense_gemm(ctx.handle, M, N, K, float(alpha), _ptr(A), A.stride(0), _ptr(B), B.stride(0),
                                      float(beta), _ptr(Cout), Cout.stride(0), int(bool(split)), C.c_void_p(stream)))
    return Cout


def dense_inverse(ctx: Context, Cm: torch.Tensor, precision: str = "fp64", stream=None) -> torch.Tensor:
    """C^{-1} of a dense square FP64 device matrix by the library's Gauss-Jordan inversion (the
    capacitance inverse of the Woodbury preconditioner); precision "mixed" computes in FP32."""
    lib = ctx.lib
    if Cm.dim() != 2 or Cm.shape[0] != Cm.shape[1] or Cm.dtype != torch.float64 or not Cm.is_cuda:
        raise ValueError("expected a square float64 CUDA matrix")
    Cm = Cm.contiguous()
    out = torch.empty_like(Cm)
    if stream is None:
        stream = torch.cuda.current_stream(Cm.device).cuda_stream
    _check(lib, lib.ncpadj_dense_inverse(ctx.handle, Cm.shape[0], _ptr(Cm), _ptr(out), PRECISION[precision],
                                         C.c_void_p(stream)))
    return out
