"""Timing harness of the oracle adjoint: the CPU baseline reported beside the GPU numbers.

Test infrastructure (oracle): run by ``bench.py`` in a child process pinned to one thread.
It times ``Step.adjoint`` as it stands -- explicit assembly of script_A, direct sparse LU of
script_A^T, all contractions -- on the beam-on-incline workload (40x10x10 cells, 20,000 tets,
451 contacts).  The state is the oracle's own start point of the step (inertial prediction
with the contact vertices lifted, multipliers from the exact local contact solve): the work
of an adjoint does not depend on how well the state was converged, and the oracle's full
forward solve of this scene takes about a minute.

    python -m oracle.timing --steps K --warmup W   ->  one JSON line on stdout
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


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--steps", type=int, default=3)
    ap.add_argument("--warmup", type=int, default=1)
    a = ap.parse_args()
    st, s, q_prev, dq, dv = beam_case()
    for _ in range(a.warmup):
        st.adjoint(s, q_prev, dq, dv)
    times = []
    for _ in range(a.steps):
        t0 = time.perf_counter()
        st.adjoint(s, q_prev, dq, dv)
        times.append(time.perf_counter() - t0)
    print(json.dumps({"seconds": times, "threads": int(os.environ.get("OMP_NUM_THREADS", "0") or 0),
                      "n_tets": st.mesh.n_tets, "n_contacts": st.nc}))


if __name__ == "__main__":
    main()
