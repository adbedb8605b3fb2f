"""Autotuner for the adjoint's launch shapes and runtime choices on a given scene.

Two stages, both timed with the real call on the real inputs:

1. The launch shape of the dominant kernels, the product with A^{-1} = P^T S^T S P: the chunk length
   (128, 256 or 512 nonzeros per warp, ``Scene.set_chunk``).  Which is fastest depends on the
   factor's row lengths and on whether S and S^T stay in L2.  ``tune_shape`` times each candidate
   and keeps the fastest.
2. The options: the precision variant (plain FP64; FP32 matrix and preconditioner with the
   capacitance inverted in FP64, by pivoted Gauss-Jordan in FP32, by the tensor-core blocked
   Gauss-Jordan, or by the tensor-core inverse refined against the FP64 capacitance), the GMRES
   restart length and the largest capacitance block inverted directly (beyond it the contact-space
   system is solved iteratively, Sec. 4.4).  Candidates whose gradients leave a relative error bound
   of the plain FP64 result on the same inputs are dropped; the fastest of the rest wins.

Choices are cached per scene signature (sizes, rounded to powers of two), so a rollout or a batch
tunes once.  Only host-side selection lives here; every timed step runs in the library's kernels.
"""
from __future__ import annotations

import json
import math
import os
from dataclasses import dataclass, field
from typing import Callable, Dict, Iterable, List, Optional, Sequence, Tuple

PRECISION_VARIANTS = (("fp64", "fp64"), ("mixed", "fp64"), ("mixed", "mixed"), ("mixed", "tf32x3"),
                      ("mixed", "refined"))
CHUNKS = (128, 256, 512)
GRAD_KEYS = ("dL_dq_prev", "dL_dv_prev", "dL_dfext", "dL_dE", "dL_dnu", "dL_dmu", "dL_dmu_contact")


@dataclass
class Trial:
    """One timed candidate."""
    options: Dict[str, object]
    ms: float                    # median time per call
    rel_err: float               # max over gradients of ||g - g_fp64|| / ||g_fp64||
    iterations: int = 0
    error: Optional[str] = None  # the call failed (not converged, unsupported, ...)


@dataclass
class Choice:
    options: Dict[str, object]
    ms: float
    rel_err: float
    trials: List[Trial] = field(default_factory=list)
    chunk: Optional[int] = None                        # launch shape of the A^{-1} product
    chunk_ms: Dict[int, float] = field(default_factory=dict)


def default_candidates(n_contacts: int, restarts: Sequence[int] = (32, 64, 128)) -> List[Dict[str, object]]:
    """Every precision variant x restart length, and for scenes with many contacts also a smaller
    direct capacitance block (an inner iterative solve around blocks of 1,024 contacts)."""
    blocks = [0] + ([1024] if n_contacts > 1024 else [])
    out = []
    for prec, cap in PRECISION_VARIANTS:
        for m in restarts:
            for cb in blocks:
                out.append({"precision": prec, "cap_precision": cap, "restart": int(m), "cap_block": int(cb)})
    return out


def tune_shape(apply: Callable[[object], None], measure: Callable[[], float], shapes: Sequence[object]):
    """Launch-shape stage: for each shape, ``apply(shape)`` then ``measure() -> ms``; the fastest shape is
    applied again and returned with every timing ({shape: ms}; a failing shape gets inf)."""
    times = {}
    for sh in shapes:
        try:
            apply(sh)
            times[sh] = float(measure())
        except Exception:  # noqa: BLE001 -- a shape that fails is skipped
            times[sh] = math.inf
    ok = [sh for sh in shapes if math.isfinite(times[sh])]
    if not ok:
        raise ValueError("no launch shape could be timed")
    best = ok[0]
    for sh in ok[1:]:
        if times[sh] < times[best]:
            best = sh
    apply(best)
    return best, times


def select(trials: Iterable[Trial], max_rel_err: float) -> Trial:
    """The fastest successful trial within the error bound; ties go to the earlier trial.
    Raises ValueError if none qualifies."""
    ok = [t for t in trials if t.error is None and t.rel_err <= max_rel_err and math.isfinite(t.ms)]
    if not ok:
        raise ValueError("no candidate met the accuracy bound")
    best = ok[0]
    for t in ok[1:]:
        if t.ms < best.ms:
            best = t
    return best


def tune(measure: Callable[[Dict[str, object]], Tuple[float, Dict[str, object], int]],
         candidates: Sequence[Dict[str, object]], reference: Dict[str, object], max_rel_err: float = 1e-3,
         norm: Callable = None) -> Choice:
    """Time every candidate with ``measure(options) -> (ms, grads, iterations)`` and pick with
    ``select``.  ``reference`` holds the plain FP64 gradients of the same inputs; ``norm`` is the
    vector norm used for the relative errors (default: Euclidean over the flattened values)."""
    if norm is None:
        def norm(x):
            return float(sum(float(v) * float(v) for v in _flat(x)) ** 0.5)
    trials = []
    for opts in candidates:
        try:
            ms, grads, iters = measure(opts)
            err = 0.0
            for k, ref in reference.items():
                if k not in grads:
                    continue
                den = norm(ref)
                diff = norm(_sub(grads[k], ref))
                err = max(err, diff / den if den > 0 else diff)
            trials.append(Trial(dict(opts), float(ms), err, int(iters)))
        except Exception as e:  # noqa: BLE001 -- a failing candidate is recorded and skipped
            trials.append(Trial(dict(opts), math.inf, math.inf, 0, f"{type(e).__name__}: {e}"))
    best = select(trials, max_rel_err)
    return Choice(best.options, best.ms, best.rel_err, trials)


def _flat(x):
    if hasattr(x, "detach"):
        return x.detach().reshape(-1).double().cpu().tolist()
    if isinstance(x, (list, tuple)):
        out = []
        for v in x:
            out.extend(_flat(v))
        return out
    return [x]


def _sub(a, b):
    if hasattr(a, "detach"):
        return a - b
    return [x - y for x, y in zip(_flat(a), _flat(b))]


def signature(n_verts: int, n_tets: int, n_contacts: int, n_scenes: int = 1) -> str:
    """Cache key: sizes rounded up to powers of two (scenes of similar size share a choice)."""
    def p2(n):
        return 0 if n <= 0 else 1 << (int(n) - 1).bit_length()
    return f"v{p2(n_verts)}-t{p2(n_tets)}-c{p2(n_contacts)}-s{int(n_scenes)}"


class Cache:
    """Choices by signature, optionally persisted as JSON."""

    def __init__(self, path: Optional[str] = None):
        self.path = path
        self.entries: Dict[str, Dict[str, object]] = {}
        if path and os.path.exists(path):
            with open(path) as f:
                self.entries = json.load(f)

    def get(self, key: str) -> Optional[Dict[str, object]]:
        e = self.entries.get(key)
        return None if e is None else dict(e["options"])

    def put(self, key: str, choice: Choice) -> None:
        opts = dict(choice.options)
        if choice.chunk is not None:
            opts["chunk"] = int(choice.chunk)
        self.entries[key] = {"options": opts, "ms": choice.ms, "rel_err": choice.rel_err}
        if self.path:
            tmp = self.path + ".tmp"
            with open(tmp, "w") as f:
                json.dump(self.entries, f, indent=1, sort_keys=True)
            os.replace(tmp, self.path)


def tune_adjoint(scene, contacts, q, q_prev, lam, dL_dq, dL_dv=None, *, eps=1e-4, rtol=1e-8,
                 candidates: Optional[Sequence[Dict[str, object]]] = None, max_rel_err: float = 1e-3,
                 repeats: int = 3, cache: Optional[Cache] = None, stream=None,
                 chunks: Optional[Sequence[int]] = CHUNKS) -> Choice:
    """Tune the launch shape and then the ``adjoint_step`` options on these inputs (device tensors, as
    for adjoint_step).

    Each timing runs the call once untimed, then ``repeats`` times between CUDA events on the call's
    stream, and takes the median.  The chunk length is timed with the FP32 tensor-core variant and left
    set on the scene (``chunks=None`` skips that stage); the returned options go straight into
    adjoint_step (``restart``, ``precision``, ``cap_precision``, ``cap_block``)."""
    import torch

    from .binding import adjoint_step
    nc = contacts.n if contacts is not None else 0
    key = signature(scene.n_verts, scene.n_tets, nc, scene.info().get("n_scenes", 1))
    if cache is not None:
        hit = cache.get(key)
        if hit is not None:
            ch = hit.pop("chunk", None)
            if ch is not None:
                scene.set_chunk(int(ch))
            return Choice(hit, float("nan"), float("nan"), chunk=ch)
    dev = q.device
    st = torch.cuda.Stream(dev) if stream is None else stream

    def call(opts):
        return adjoint_step(scene, contacts, q, q_prev, lam, dL_dq, dL_dv, eps=eps, rtol=rtol,
                            precision=opts["precision"], cap_precision=opts["cap_precision"],
                            restart=int(opts["restart"]), cap_block=int(opts["cap_block"]), stream=st.cuda_stream)

    with torch.cuda.stream(st):
        ref, _ = call({"precision": "fp64", "cap_precision": "fp64", "restart": 64, "cap_block": 0})
    torch.cuda.synchronize(dev)
    reference = {k: ref[k].clone() for k in GRAD_KEYS if k in ref}

    def measure(opts):
        with torch.cuda.stream(st):
            call(opts)
            times = []
            grads = stats = None
            for _ in range(max(1, repeats)):
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(st)
                grads, stats = call(opts)
                e1.record(st)
                e1.synchronize()
                times.append(e0.elapsed_time(e1))
        times.sort()
        return times[len(times) // 2], grads, stats["iterations"]

    chunk, chunk_ms = None, {}
    if chunks:
        # timed with the tensor-core variant, or plain FP64 where that one fails on the scene; a scene on
        # which neither runs keeps its chunk length
        before = getattr(scene, "chunk", None)
        for base in ({"precision": "mixed", "cap_precision": "tf32x3", "restart": 64, "cap_block": 0},
                     {"precision": "fp64", "cap_precision": "fp64", "restart": 64, "cap_block": 0}):
            try:
                chunk, chunk_ms = tune_shape(scene.set_chunk, lambda b=base: measure(b)[0], list(chunks))
                break
            except ValueError:
                chunk, chunk_ms = None, {}
        if chunk is None and before is not None:
            scene.set_chunk(before)
    choice = tune(measure, candidates or default_candidates(nc), reference, max_rel_err,
                  norm=lambda x: float(torch.linalg.norm(x.double() if hasattr(x, "double") else torch.tensor(x))))
    choice.chunk, choice.chunk_ms = chunk, chunk_ms
    if cache is not None:
        cache.put(key, choice)
    return choice


__all__ = ["Trial", "Choice", "Cache", "default_candidates", "select", "tune", "tune_adjoint", "tune_shape",
           "signature", "PRECISION_VARIANTS", "CHUNKS"]
