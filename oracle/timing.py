"""Timing harness of the oracle adjoint: the CPU baseline reported beside the GPU numbers.

Test infrastructure (oracle): run by ``bench.py`` in a child process pinned to one thread.
It times ``Step.adjoint`` as it stands -- explicit assembly of script_A, direct sparse LU of
script_A^T, all contractions -- on the beam-on-incline workload (40x10x10 cells, 20,000 tets,
451 contacts).  The state is either the oracle's own start point of the step (inertial
prediction with the contact vertices lifted, multipliers from the exact local contact solve)
-- the work of an adjoint does not depend on how well the state was converged, and the
oracle's full forward solve of this scene takes about a minute -- or, with ``--state``, a
state given in an .npz file (q, q_prev, the seeds dL_dq, dL_dv; multipliers again from the
exact local solve at q).  Gradients stored in that file as ``<variant>/<key>`` are compared
with the oracle's, and their relative errors are reported.

    python -m oracle.timing --steps K --warmup W [--state file.npz]  ->  one JSON line on stdout
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


# the GPU output names and the oracle's, for the comparison
KEYS = (("dL_dq_prev", "dL_dq_prev"), ("dL_dv_prev", "dL_dv_prev"), ("dL_dfext", "dL_dfext"), ("z", "z"),
        ("dL_dE", "dL_dE"), ("dL_dnu", "dL_dnu"), ("dL_dmu", "dL_dmu_region"), ("dL_dmu_contact", "dL_dmu_contact"))


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    ap.add_argument("--state", default=None)
    a = ap.parse_args()
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
