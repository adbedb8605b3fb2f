"""Shared test cases: converged oracle states of the seeded scenes (cached per process)."""
from __future__ import annotations

import functools

import numpy as np

import synth
from oracle.step import Step


def make_step(scene, contacts, E=None, nu=None, eps=None, model="neo_hookean", bend=None):
    return Step(scene.X, scene.tets, scene.E if E is None else E, scene.nu if nu is None else nu,
                scene.density, scene.h, scene.gravity, contacts, scene.eps if eps is None else eps, model,
                thickness=getattr(scene, "thickness", None),
                bend=getattr(scene, "bend", 0.0) if bend is None else bend)


@functools.lru_cache(maxsize=None)
def rollout(name: str, k: int, model: str = "neo_hookean", **kw):
    """Problem, and the oracle state at the start of step k: (q_prev, v_prev) after k forward
    steps from the initial state (contacts re-detected every step) under the given model."""
    pb = getattr(synth, name)(**kw)
    sc = pb.scene
    q_prev, v_prev = pb.q0.copy(), pb.v0.copy()
    for _ in range(k):
        ct = sc.contacts(q_prev)
        st = make_step(sc, ct, model=model)
        s = st.forward(q_prev, v_prev)
        assert s.residual < 1e-8, s.residual
        v_prev = (s.q - q_prev) / sc.h
        q_prev = s.q
    return pb, q_prev, v_prev


@functools.lru_cache(maxsize=None)
def step_case(name: str, k: int, model: str = "neo_hookean", **kw):
    """(problem, Step, converged State, q_prev, v_prev) for step k of a scene's rollout."""
    pb, q_prev, v_prev = rollout(name, k, model, **kw)
    sc = pb.scene
    ct = sc.contacts(q_prev)
    st = make_step(sc, ct, model=model)
    s = st.forward(q_prev, v_prev)
    assert s.residual < 1e-8, s.residual
    return pb, st, s, q_prev, v_prev


def rel(a, b):
    a = np.asarray(a, float)
    b = np.asarray(b, float)
    return np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-30)
