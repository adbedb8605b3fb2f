"""Timing harness of the oracle adjoint: the CPU baseline reported beside the GPU numbers.

Test infrastructure (oracle): run by ``bench.py`` in a child process pinned to one thread.
It times ``Step.adjoint`` as it stands -- explicit assembly of script_A, direct sparse LU of
script_A^T, all contractions -- on one of two workloads:

* the beam on the incline (40x10x10 cells, 20,000 tets, 451 contacts);
* with ``--batch``, the 64 uneven blocks of the batched workload, of which a seeded sample of
  ``BATCH_SAMPLE`` blocks is timed (one adjoint per block; the mean over the sample stands in
  for the mean block of the batch).

The state is either the oracle's own start point of the step (inertial prediction with the
contact vertices lifted, multipliers from the exact local contact solve) -- the work of an
adjoint does not depend on how well the state was converged -- or, with ``--state``, a state
given in an .npz file (q, q_prev, the seeds dL_dq, dL_dv, under ``b<i>/`` per block in batch
mode; multipliers again from the exact local solve at q).  Gradients stored in that file as
``<variant>/<key>`` (``b<i>/<variant>/<key>``) are compared with the oracle's, and their
relative errors are reported.

    python -m oracle.timing [--batch] --steps K --warmup W [--state file.npz]  ->  one JSON line
"""
from __future__ import annotations

import argparse
import json
import os
import sys
import time

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import synth  # noqa: E402
from oracle.step import State, Step  # noqa: E402


def beam_case():
    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    st = Step(sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h, sc.gravity, ct, sc.eps)
    qt = st.qtilde(pb.q0, pb.v0, np.zeros_like(pb.q0))
    q = st.start_point(pb.q0, qt)
    lam_n, gam = st.local_multipliers(q, pb.q0)
    rng = np.random.default_rng(0)
    return st, State(q, lam_n, gam), pb.q0, rng.normal(size=q.shape), rng.normal(size=q.shape) * 1e-3


def state_case(path):
    """The beam at a given state (see the module docstring); also returns the stored gradients."""
    d = np.load(path)
    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    st = Step(sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h, sc.gravity, ct, sc.eps)
    q, q_prev = d["q"], d["q_prev"]
    lm = st.local_multipliers(q, q_prev)
    if lm is None:
        raise ValueError("the given state is outside the local contact solve's domain")
    grads = {}
    for k in d.files:
        if "/" in k:
            variant, key = k.split("/", 1)
            grads.setdefault(variant, {})[key] = d[k]
    return st, State(q, lm[0], lm[1]), q_prev, d["dL_dq"], d["dL_dv"], grads


BATCH_SAMPLE = 8
_BLOCKS = None


def batch_sample_ids(n_blocks: int = 64, k: int = BATCH_SAMPLE, seed: int = 0):
    """The blocks of the batched workload whose oracle adjoints are timed (seeded, sorted)."""
    return sorted(int(i) for i in np.random.default_rng(seed).choice(n_blocks, k, replace=False))


def block_case(i, state=None):
    """Block i of the 64-block batch: (Step, State, q_prev, dL_dq, dL_dv, stored gradients).  The
    contact set is detected at the block's start state, as the GPU bench does."""
    global _BLOCKS
    if _BLOCKS is None:
        _BLOCKS = synth.block_batch(64)
    pb = _BLOCKS[i]
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    st = Step(sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h, sc.gravity, ct, sc.eps)
    grads = {}
    if state is None:
        qt = st.qtilde(pb.q0, pb.v0, np.zeros_like(pb.q0))
        q = st.start_point(pb.q0, qt)
        q_prev = pb.q0
        rng = np.random.default_rng(100 + i)
        dq, dv = rng.normal(size=q.shape), rng.normal(size=q.shape) * 1e-3
    else:
        d = state
        pre = f"b{i}/"
        q, q_prev, dq, dv = d[pre + "q"], d[pre + "q_prev"], d[pre + "dL_dq"], d[pre + "dL_dv"]
        for k in d.files:
            if k.startswith(pre) and k.count("/") == 2:
                _, variant, key = k.split("/")
                grads.setdefault(variant, {})[key] = d[k]
    lm = st.local_multipliers(q, q_prev)
    if lm is None:
        raise ValueError(f"block {i}: the state is outside the local contact solve's domain")
    return st, State(q, lm[0], lm[1]), q_prev, dq, dv, grads


def batch_main(a):
    ids = batch_sample_ids()
    given = np.load(a.state) if a.state else None
    cases = [block_case(i, given) for i in ids]
    out = None
    for _ in range(a.warmup):
        st, s, q_prev, dq, dv, _ = cases[0]
        out = st.adjoint(s, q_prev, dq, dv)
    times, errs, blocks = [], {}, []
    n = len(cases) if given is not None else a.steps
    for k in range(n):
        st, s, q_prev, dq, dv, g = cases[k % len(cases)]
        t0 = time.perf_counter()
        out = st.adjoint(s, q_prev, dq, dv)
        times.append(time.perf_counter() - t0)
        blocks.append({"block": ids[k % len(cases)], "n_tets": st.mesh.n_tets, "n_contacts": st.nc})
        for variant, gv in g.items():
            e = errs.get(variant, 0.0)
            for key, ok in KEYS:
                if key in gv and not (st.nc == 0 and ok in ("dL_dmu_region", "dL_dmu_contact")):
                    ref = np.asarray(out[ok]).reshape(-1)
                    e = max(e, float(np.linalg.norm(np.asarray(gv[key]).reshape(-1) - ref) /
                                     max(np.linalg.norm(ref), 1e-300)))
            errs[variant] = e
    print(json.dumps({"seconds": times, "threads": int(os.environ.get("OMP_NUM_THREADS", "0") or 0),
                      "blocks": blocks, "state": "given" if given is not None else "start point",
                      "rel_err_vs_oracle": errs}))


# the GPU output names and the oracle's, for the comparison
KEYS = (("dL_dq_prev", "dL_dq_prev"), ("dL_dv_prev", "dL_dv_prev"), ("dL_dfext", "dL_dfext"), ("z", "z"),
        ("dL_dE", "dL_dE"), ("dL_dnu", "dL_dnu"), ("dL_dmu", "dL_dmu_region"), ("dL_dmu_contact", "dL_dmu_contact"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--state", default=None)
    ap.add_argument("--batch", action="store_true", help="the 64-block batched workload (a seeded sample of blocks)")
    a = ap.parse_args()
    if a.batch:
        return batch_main(a)
    if a.state:
        st, s, q_prev, dq, dv, given = state_case(a.state)
    else:
        (st, s, q_prev, dq, dv), given = beam_case(), {}
    out = None
    for _ in range(a.warmup):
        out = st.adjoint(s, q_prev, dq, dv)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        out = st.adjoint(s, q_prev, dq, dv)
        times.append(time.perf_counter() - t0)
    errs = {}
    for variant, g in given.items():
        e = 0.0
        for key, ok in KEYS:
            if key in g:
                ref = np.asarray(out[ok]).reshape(-1)
                e = max(e, float(np.linalg.norm(np.asarray(g[key]).reshape(-1) - ref) / max(np.linalg.norm(ref), 1e-300)))
        errs[variant] = e
    print(json.dumps({"seconds": times, "threads": int(os.environ.get("OMP_NUM_THREADS", "0") or 0),
                      "n_tets": st.mesh.n_tets, "n_contacts": st.nc, "state": "given" if a.state else "start point",
                      "rel_err_vs_oracle": errs}))


if __name__ == "__main__":
    main()
