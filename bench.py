"""Benchmark: adjoint gradients/s of one implicit step on the beam-on-incline scene.

Workload (the mid-size single scene): Neo-Hookean beam of 40x10x10 hex cells x 5 tets (20,000 tets,
4,961 vertices), E=5e5, nu=0.45, rho=1000, resting on a 20 deg plane with mu=0.3 (451 frictional
contacts, eps=1e-4), h=1/100.  The state is produced on the GPU by the forward step (3 steps from
rest, so the beam slides); one bench step = one complete adjoint step through the C-ABI: assembly
of script_A^T (per-tet SVD Jacobians, contact blocks), Woodbury set-up (Delassus, capacitance,
its inversion), GMRES to rtol 1e-8 and all gradient contractions (dL/dqbar, dL/dvbar, dL/dfext,
dL/dE, dL/dnu per tet, dL/dmu).

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]

Prints one JSON line.  Timing: W untimed warm-up steps, then K steps, each bracketed by CUDA
events on the library's stream; L2 (129 MB) is flushed by writing a 512 MB buffer before every
timed step (the working set, ~90 MB, would otherwise stay resident).  Multi-GPU: the path does
not shard within a scene, so N ranks run N independent replicas (one process per GPU); value is
the adjoints of all ranks over the slowest rank's time.
"""
from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

METRIC = "adjoint gradients/sec per step (batched FP32/64 vs plain FP64) at rel err <=1e-3"
WORKLOAD = ("beam 40x10x10 cells x 5 tets (20000 tets, 4961 verts), 451 frictional contacts on a 20deg incline, "
            "mu=0.3, eps=1e-4, h=1/100, one adjoint step (state: GPU forward, 3 steps from rest)")


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    if os.path.exists(p):
        d = json.load(open(p))
        return d.get("hbm_gbs", 6777.0), "measured"
    return 6800.0, "fallback"


# --------------------------------------------------------------------------------------------
# clocks sampled during the timed region
# --------------------------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, device_index=0):
        self.dev = device_index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", f"--id={self.dev}", f"--query-gpu={self.FIELDS}",
                                          "--format=csv,noheader,nounits", "-lms", "100"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            parts = [x.strip() for x in ln.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for nm, val in zip(names, parts[5:9]):
                if val.lower().startswith("active"):
                    reasons.add(nm)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


# --------------------------------------------------------------------------------------------
# reference arm and CPU baseline: the FP64 oracle, single-threaded, in a child process
# --------------------------------------------------------------------------------------------
def oracle_times(steps, warmup, state=None):
    env = dict(os.environ, OMP_NUM_THREADS="1", OPENBLAS_NUM_THREADS="1", MKL_NUM_THREADS="1",
               CUDA_VISIBLE_DEVICES="")
    cmd = [sys.executable, "-m", "oracle.timing", "--steps", str(steps), "--warmup", str(warmup)]
    if state:
        cmd += ["--state", state]
    r = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=900)
    if r.returncode != 0:
        raise RuntimeError(r.stderr[-2000:])
    return json.loads(r.stdout.strip().splitlines()[-1])


def models_leg(pkg, torch, dev, scene, n_verts, q_adj, timed):
    """The co-rotational and ARAP adjoints, then 40 stiff bindings on Neo-Hookean tets, on the
    bench's scene at its state.  ``timed(**kw) -> (total ms, stats list)`` times the headline
    variant.  Failures are reported in the result, and the scene is left Neo-Hookean."""
    res = {}
    try:
        for mname in ("corotational", "arap"):
            scene.set_model(mname)
            tm, sm = timed()
            res[mname] = {"gradients_per_s": len(sm) / (tm / 1e3),
                          "krylov_iterations": statistics.median(x["iterations"] for x in sm),
                          "ms_assemble": statistics.mean(x["ms_assemble"] for x in sm)}
        scene.set_model("neo_hookean")
        nbind = 40  # vertices spread over the mesh, held where they are by stiff springs
        bv = torch.arange(0, n_verts, max(1, n_verts // nbind), device=dev, dtype=torch.int32)[:nbind].contiguous()
        nbind = int(bv.shape[0])
        bd = pkg.Bindings(bv, q_adj[bv.long()].contiguous(), torch.full((nbind,), 1e-6, dtype=torch.float64, device=dev))
        tm, sm = timed(bindings=bd)
        res["bindings"] = {"n": nbind, "compliance": 1e-6, "gradients_per_s": len(sm) / (tm / 1e3),
                           "krylov_iterations": statistics.median(x["iterations"] for x in sm)}
    except Exception as e:  # noqa: BLE001
        res["error"] = str(e)[:300]
    try:
        scene.set_model("neo_hookean")
    except Exception as e:  # noqa: BLE001
        res["error"] = res.get("error", "") + f"; reset: {str(e)[:100]}"
    return res


def cpu_baseline_leg(arrays):
    """The oracle at the bench's state: ``arrays`` holds q, q_prev, dL_dq, dL_dv and the GPU
    gradients as '<variant>/<key>'.  Falls back to the oracle's own start point if that state
    cannot be used.  Returns (the cpu_baseline object, the relative errors vs the oracle or None)."""
    import tempfile
    d, err, where = None, None, "the bench's GPU state (3 forward steps from rest, same seeds)"
    try:
        with tempfile.TemporaryDirectory() as tdir:
            path = os.path.join(tdir, "state.npz")
            np.savez(path, **arrays)
            d = oracle_times(3, 1, state=path)
        err = d.get("rel_err_vs_oracle")
    except Exception:  # noqa: BLE001 -- fall back to the oracle's own start point
        where = "the oracle's start point of step 1"
        try:
            d = oracle_times(3, 1)
        except Exception as e:  # noqa: BLE001
            return {"value": None, "unit": "gradients/s", "cores": 1, "kind": "oracle", "sample": f"failed: {e}"}, None
    return ({"value": len(d["seconds"]) / sum(d["seconds"]), "unit": "gradients/s", "cores": d["threads"],
             "kind": "oracle", "sample": f"{len(d['seconds'])} oracle adjoints of the beam (assembly + direct sparse "
             f"LU + contractions) at {where}, after 1 warm-up"}, err)


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    d = oracle_times(args.steps, args.warmup)
    secs = d["seconds"]
    total = sum(secs)
    val = len(secs) / total
    sample = (f"{len(secs)} oracle adjoints (explicit assembly + direct sparse LU + contractions) of the beam "
              f"at the oracle's start point of step 1, {d['threads']} thread")
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": val, "unit": "gradients/s", "n_gpus": args.gpus,
        "steps": len(secs), "warmup": args.warmup, "ms_per_step": 1e3 * total / len(secs), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": WORKLOAD},
        "cpu_baseline": {"value": val, "unit": "gradients/s", "cores": d["threads"], "kind": "oracle", "sample": sample},
        "e2e": {"value": val, "unit": "gradients/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }))


# --------------------------------------------------------------------------------------------
# batched uneven scenes: 64 independent blocks (log-uniform 2k..50k tets), one adjoint each
# --------------------------------------------------------------------------------------------
def apply_roofline(pkg, torch, dev, scene, K):
    """GB/s of the product with A^{-1} = P^T S^T S P (two k_spmv_chunks launches, FP64, 3 RHS) on a
    scene: K applies captured into one CUDA graph and replayed, timed with events on the replay
    stream.  Returns algorithmic bytes (Cholesky-factor based) and the kernels' own bytes (S, S^T)."""
    info = scene.info()
    n3 = 3 * scene.n_verts
    sx = torch.randn(scene.n_verts, 3, dtype=torch.float64, device=dev)
    sy = torch.empty_like(sx)
    sst = torch.cuda.Stream(dev)
    for _ in range(3):
        pkg.elastic_solve(scene, sx, sy, stream=sst.cuda_stream)
    torch.cuda.synchronize(dev)
    g = torch.cuda.CUDAGraph()
    with torch.cuda.graph(g, stream=sst):
        for _ in range(K):
            pkg.elastic_solve(scene, sx, sy, stream=torch.cuda.current_stream().cuda_stream)
    with torch.cuda.stream(sst):
        g.replay()
        torch.cuda.synchronize(dev)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(sst)
        for _ in range(3):
            g.replay()
        e1.record(sst)
    torch.cuda.synchronize(dev)
    ms = e0.elapsed_time(e1) / (3 * K)
    alg = 2 * info["nnz_L"] * 12 + 4 * n3 * 8
    kb = 2 * info["nnz_Linv"] * 12 + 4 * n3 * 8
    peak, src = peaks()
    return {"kernel": "k_spmv_chunks x2 (A^-1 = P^T S^T S P, FP64, 3 RHS)", "bound": "hbm",
            "achieved": alg / (ms / 1e3) / 1e9, "peak": peak, "unit": "GB/s",
            "frac": alg / (ms / 1e3) / 1e9 / peak, "traffic": None, "peak_source": src, "ms_per_launch_pair": ms,
            "algorithmic_bytes": alg, "kernel_bytes": kb, "kernel_bytes_gbs": kb / (ms / 1e3) / 1e9,
            "kernel_bytes_frac": kb / (ms / 1e3) / 1e9 / peak}


def batched(pkg, torch, dev, steps, warmup):
    import synth
    blocks = synth.block_batch(64)
    h = blocks[0].scene.h
    ctx = pkg.Context(dev.index or 0)
    t0 = time.perf_counter()
    scene = pkg.Scene.batch(ctx, [(b.scene.X, b.scene.tets, b.scene.E, b.scene.nu, b.scene.density) for b in blocks], h)
    t_build = time.perf_counter() - t0
    off = scene.vertex_offsets
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    # one forward step of every block (contacts from its start state) on the GPU gives the adjoint state
    q0 = T(np.concatenate([b.q0 for b in blocks]))
    v0 = T(np.concatenate([b.v0 for b in blocks]))
    verts, frames, dn, mu, reg = [], [], [], [], []
    for i, b in enumerate(blocks):
        ct = b.scene.contacts(b.q0)
        verts.append(ct.vertex + off[i])
        frames.append(ct.frame)
        dn.append(ct.d_n)
        mu.append(ct.mu)
        reg.append(np.full(ct.n, i, np.int32))
    nc = sum(len(v) for v in verts)
    contacts = pkg.Contacts(T(np.concatenate(verts), torch.int32), T(np.concatenate(frames)), T(np.concatenate(dn)),
                            T(np.concatenate(mu)), None, T(np.concatenate(reg), torch.int32), len(blocks))
    # impacts at up to ~0.15 m/s make some blocks' Newton solves long: the adjoint is timed at the
    # iterate reached within 150 steps, whose residual is reported
    try:
        q, lam, fs = pkg.forward_step(scene, contacts, q0, v0, None, tuple(blocks[0].scene.gravity),
                                      eps=blocks[0].scene.eps, max_newton=150, cap_precision="mixed")
    except pkg.NcpadjError as e:
        if not hasattr(e, "state"):
            raise
        (q, lam), fs = e.state, e.stats
    tgt = T(np.concatenate([b.q_target for b in blocks]))
    dq = 2 * (q - tgt)
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    res = {}
    for prec in ("fp64", "mixed"):
        for _ in range(warmup):
            pkg.adjoint_step(scene, contacts, q, q0, lam.contiguous(), dq, None, eps=blocks[0].scene.eps,
                             precision=prec, cap_precision=prec, stream=stream.cuda_stream)
        ms = []
        sts = []
        with torch.cuda.stream(stream):
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g, st = pkg.adjoint_step(scene, contacts, q, q0, lam.contiguous(), dq, None, eps=blocks[0].scene.eps,
                                         precision=prec, cap_precision=prec, stream=stream.cuda_stream)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
                sts.append(st)
        res[prec] = {"gradients_per_s": len(blocks) * steps / (sum(ms) / 1e3), "ms_per_call": sum(ms) / steps,
                     "krylov_iterations": statistics.median(x["iterations"] for x in sts),
                     "stage_ms": {k: statistics.mean(x[k] for x in sts) for k in
                                  ("ms_assemble", "ms_setup", "ms_krylov", "ms_contract")}}
        res[prec + "_grads"] = {k: v.clone() for k, v in g.items()}
    err = max(float((torch.linalg.norm(res["mixed_grads"][k] - res["fp64_grads"][k]) /
                     torch.linalg.norm(res["fp64_grads"][k]).clamp_min(1e-300)).item()) for k in res["fp64_grads"])
    for k in ("mixed_grads", "fp64_grads"):
        res.pop(k)
    info = scene.info()
    roof = apply_roofline(pkg, torch, dev, scene, 10)
    return {"workload": f"64 independent blocks, {scene.n_tets} tets / {scene.n_verts} verts in total "
                        f"(log-uniform 2k..50k tets each), {nc} contacts in {sum(1 for v in verts if len(v))} blocks, "
                        "one adjoint step of every block per call",
            "fp64": res["fp64"], "mixed": res["mixed"], "max_rel_err_mixed_vs_fp64": err,
            "scene_build_s": t_build, "nnz_Linv": info["nnz_Linv"], "forward_newton_iters": fs["newton_iters"],
            "forward_residual": fs["residual"], "roofline_Ainv": roof}


def sphere(pkg, torch, dev, steps, warmup):
    """The large contact-heavy scene at full size: ball (r = 0.1 m, ~32k vertices, ~211k tets) pressed
    between the ground and a kinematic plate, ~2,300 frictional contacts in 32 friction regions.
    One GPU forward step gives the state; the adjoint is timed in FP64 and mixed precision, and
    the Krylov iterations of Woodbury, Jacobi and no preconditioner are compared (capped at 5000)."""
    import synth
    log = lambda m: print(f"[sphere {time.strftime('%H:%M:%S')}] {m}", file=sys.stderr, flush=True)  # noqa: E731
    pb = synth.sphere_press()
    sc = pb.scene
    log(f"mesh {sc.n_verts} verts {sc.n_tets} tets")
    ctx = pkg.Context(dev.index or 0)
    t0 = time.perf_counter()
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    t_build = time.perf_counter() - t0
    log(f"scene built in {t_build:.1f} s")
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    ct = sc.contacts(pb.q0)
    contacts = pkg.Contacts(T(ct.vertex, torch.int32), T(ct.frame), T(ct.d_n), T(ct.mu), None,
                            T(ct.region, torch.int32), ct.n_regions)
    q0, v0 = T(pb.q0), T(pb.v0)
    t0 = time.perf_counter()
    try:
        q, lam, fs = pkg.forward_step(scene, contacts, q0, v0, None, tuple(sc.gravity), eps=sc.eps, max_newton=40)
    except pkg.NcpadjError as e:  # time the adjoint at the last iterate; its residual is reported
        if not hasattr(e, "state"):
            raise
        (q, lam), fs = e.state, e.stats
    t_fwd = time.perf_counter() - t0
    log(f"forward {t_fwd:.1f} s, {fs['newton_iters']} Newton iterations, residual {fs['residual']:.2e}")
    dq = 2 * (q - T(pb.q_target))
    lam = lam.contiguous()
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    out, grads = {}, {}
    for prec in ("fp64", "mixed"):
        kw = dict(eps=sc.eps, precision=prec, cap_precision="mixed", stream=stream.cuda_stream,
                  want=("dL_dfext", "dL_dmu", "z"))
        for _ in range(warmup):
            pkg.adjoint_step(scene, contacts, q, q0, lam, dq, None, **kw)
        ms, sts = [], []
        with torch.cuda.stream(stream):
            for _ in range(steps):
                flush.zero_()
                e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
                e0.record(stream)
                g, st = pkg.adjoint_step(scene, contacts, q, q0, lam, dq, None, **kw)
                e1.record(stream)
                torch.cuda.synchronize(dev)
                ms.append(e0.elapsed_time(e1))
                sts.append(st)
        out[prec] = {"gradients_per_s": steps / (sum(ms) / 1e3), "ms_per_call": sum(ms) / steps,
                     "krylov_iterations": statistics.median(x["iterations"] for x in sts),
                     "capacitance_blocks": sts[-1]["capacitance_blocks"],
                     "stage_ms": {k: statistics.mean(x[k] for x in sts) for k in
                                  ("ms_assemble", "ms_setup", "ms_krylov", "ms_contract", "ms_cap_inverse")}}
        grads[prec] = {k: v.clone() for k, v in g.items()}
        log(f"{prec}: {out[prec]['ms_per_call']:.1f} ms per adjoint, {out[prec]['krylov_iterations']} iterations")
    err = max(float((torch.linalg.norm(grads["mixed"][k] - grads["fp64"][k]) /
                     torch.linalg.norm(grads["fp64"][k]).clamp_min(1e-300)).item()) for k in grads["fp64"])
    iters = {}
    for pc in ("woodbury", "jacobi", "none"):
        try:
            _, st = pkg.adjoint_step(scene, contacts, q, q0, lam, dq, None, eps=sc.eps, precision="mixed",
                                     cap_precision="mixed", precond=pc, max_iters=5000, want=("z",))
            iters[pc] = st["iterations"]
        except pkg.NcpadjError as e:
            iters[pc] = "not converged in 5000" if "NOT_CONVERGED" in str(e) else str(e)[:120]
    info = scene.info()
    return {"workload": f"ball r=0.1 m flattened at |z|<=5 cm, {sc.n_verts} verts / {sc.n_tets} tets, "
                        f"{ct.n} frictional contacts (ground + plate pressing 0.5 mm), {ct.n_regions} friction "
                        "regions, h=1/60, E=1e5, nu=0.4",
            "fp64": out["fp64"], "mixed": out["mixed"], "max_rel_err_mixed_vs_fp64": err,
            "krylov_iterations_by_preconditioner": iters, "scene_build_s": t_build, "forward_s": t_fwd,
            "forward_newton_iters": fs["newton_iters"], "forward_residual": fs["residual"],
            "nnz_L": info["nnz_L"], "nnz_Linv": info["nnz_Linv"], "factor_ms": info["ms_factor"]}


def quadruped_measure(pkg, torch, dev, steps, warmup, scale):
    """The actuated soft quadruped (torso, four legs, foot pads; ``scale`` = 1: ~483k tets, ~129k
    vertices, ~19.9k pad contacts, mu = 0.8, h = 1/200) with seeded per-tet activations: one GPU
    forward step gives the state, then the one-step adjoint with dL/da is timed (mixed precision,
    Woodbury with the inner capacitance solve) and the Krylov iterations of Woodbury and of the
    elastic-only preconditioner are compared."""
    import synth
    log = lambda m: print(f"[quadruped {time.strftime('%H:%M:%S')}] {m}", file=sys.stderr, flush=True)  # noqa: E731
    s = float(scale)
    kw = {} if s == 1.0 else dict(torso=(max(2, round(120 * s)), max(2, round(80 * s)), max(1, round(5 * s))),
                                  leg_r=max(1.5, 8 * s), leg_h=max(2, round(12 * s)),
                                  leg_c=(max(2, round(50 * s)), max(2, round(32 * s))),
                                  pad=(max(2, round(78 * s)), max(2, round(62 * s)), max(1, round(2 * s))),
                                  cell=5e-3 / s)
    pb = synth.quadruped(**kw)
    sc = pb.scene
    log(f"mesh {sc.n_verts} verts {sc.n_tets} tets")
    ctx = pkg.Context(dev.index or 0)
    t0 = time.perf_counter()
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    scene.set_fibres(pb.fibre)
    t_build = time.perf_counter() - t0
    log(f"scene built in {t_build:.1f} s")
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    ct = sc.contacts(pb.q0)
    contacts = pkg.Contacts(T(ct.vertex, torch.int32), T(ct.frame), T(ct.d_n), T(ct.mu), None,
                            T(ct.region, torch.int32), ct.n_regions)
    q0, v0 = T(pb.q0), T(pb.v0)
    act = T(pb.act, torch.float32)
    t0 = time.perf_counter()
    try:
        q, lam, fs = pkg.forward_step(scene, contacts, q0, v0, None, tuple(sc.gravity), eps=sc.eps, max_newton=30,
                                      act=act)
    except pkg.NcpadjError as e:
        if not hasattr(e, "state"):
            raise
        (q, lam), fs = e.state, e.stats
    t_fwd = time.perf_counter() - t0
    log(f"forward {t_fwd:.1f} s, {fs['newton_iters']} Newton iterations, residual {fs['residual']:.2e}")
    dq = torch.zeros_like(q)
    dq[:, 0] = -1.0 / q.shape[0]  # L = -mean x
    lam = lam.contiguous()
    stream = torch.cuda.Stream(dev)
    akw = dict(eps=sc.eps, precision="mixed", cap_precision="mixed", stream=stream.cuda_stream,
               want=("dL_dact", "dL_dmu", "z"))
    for _ in range(warmup):
        pkg.adjoint_step(scene, contacts, q, q0, lam, dq, None, **akw)
    ms, sts = [], []
    with torch.cuda.stream(stream):
        for _ in range(steps):
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            g, st = pkg.adjoint_step(scene, contacts, q, q0, lam, dq, None, **akw)
            e1.record(stream)
            torch.cuda.synchronize(dev)
            ms.append(e0.elapsed_time(e1))
            sts.append(st)
    log(f"adjoint {sum(ms) / len(ms):.1f} ms, {sts[-1]['iterations']} iterations, inner {sts[-1]['inner_iterations']}")
    iters = {}
    for pc in ("woodbury", "elastic"):
        try:
            _, st = pkg.adjoint_step(scene, contacts, q, q0, lam, dq, None, eps=sc.eps, precision="mixed",
                                     cap_precision="mixed", precond=pc, max_iters=2000, want=("z",))
            iters[pc] = st["iterations"]
        except pkg.NcpadjError as e:
            iters[pc] = "not converged in 2000" if "NOT_CONVERGED" in str(e) else str(e)[:120]
        log(f"iterations {pc}: {iters[pc]}")
    info = scene.info()
    return {"workload": f"soft quadruped, {sc.n_verts} verts / {sc.n_tets} tets, {ct.n} pad contacts (mu=0.8), "
                        "per-tet activations N(0, 1e3) Pa, h=1/200, one adjoint step with dL/da (mixed)",
            "gradients_per_s": steps / (sum(ms) / 1e3), "ms_per_call": sum(ms) / steps,
            "krylov_iterations": statistics.median(x["iterations"] for x in sts),
            "inner_iterations": statistics.median(x["inner_iterations"] for x in sts),
            "capacitance_blocks": sts[-1]["capacitance_blocks"],
            "stage_ms": {k: statistics.mean(x[k] for x in sts) for k in
                         ("ms_assemble", "ms_setup", "ms_krylov", "ms_contract", "ms_cap_inverse")},
            "krylov_iterations_by_preconditioner": iters, "scene_build_s": t_build, "forward_s": t_fwd,
            "forward_newton_iters": fs["newton_iters"], "forward_residual": fs["residual"],
            "nnz_L": info["nnz_L"], "nnz_Linv": info["nnz_Linv"], "factor_ms": info["ms_factor"]}


# --------------------------------------------------------------------------------------------
# our arm
# --------------------------------------------------------------------------------------------
def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=20)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--precision", default="fp64", choices=["fp64"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-e2e", action="store_true", help="skip the host-buffer end-to-end leg (profiling runs)")
    ap.add_argument("--no-batch", action="store_true", help="skip the batched 64-block measurement")
    ap.add_argument("--no-models", action="store_true",
                    help="skip the co-rotational / ARAP / bindings timings on the beam")
    ap.add_argument("--sphere", action="store_true", help="add the large contact-heavy sphere measurement")
    ap.add_argument("--quadruped", action="store_true", help="add the actuated quadruped measurement")
    ap.add_argument("--quad-scale", type=float, default=1.0, help="linear scale of the quadruped (1 = full size)")
    ap.add_argument("--roofline-only", choices=["beam", "batched"], default=None,
                    help="build the scene and run only the A^-1 roofline measurement (for profiler captures)")
    args = ap.parse_args()
    if args.impl == "reference":
        return run_reference(args)

    import torch
    import torch.distributed as dist

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1:
        dist.init_process_group("nccl")
    torch.cuda.set_device(local)
    dev = torch.device("cuda", local)

    import __graft_entry__ as g
    g.build()
    import paper_2603_16478_gb300 as pkg
    import synth

    if args.roofline_only:
        ctx = pkg.Context(local)
        if args.roofline_only == "beam":
            b = synth.beam_incline().scene
            scene = pkg.Scene(ctx, b.X, b.tets, b.E, b.nu, b.density, b.h)
        else:
            blocks = synth.block_batch(64)
            scene = pkg.Scene.batch(ctx, [(x.scene.X, x.scene.tets, x.scene.E, x.scene.nu, x.scene.density)
                                          for x in blocks], blocks[0].scene.h)
        print(json.dumps({"roofline_only": args.roofline_only, "roofline": apply_roofline(pkg, torch, dev, scene, 10)}))
        return

    pb = synth.beam_incline()
    sc = pb.scene
    ct = sc.contacts(pb.q0)
    ctx = pkg.Context(local)
    scene = pkg.Scene(ctx, sc.X, sc.tets, sc.E, sc.nu, sc.density, sc.h)
    T = lambda a, dt=torch.float64: torch.as_tensor(np.ascontiguousarray(a), dtype=dt, device=dev)  # noqa: E731
    contacts = pkg.Contacts(T(ct.vertex, torch.int32), T(ct.frame), T(ct.d_n), T(ct.mu), None,
                            T(ct.region, torch.int32), ct.n_regions)
    # converged state from the GPU forward step: 3 steps from rest
    q_prev, v_prev = T(pb.q0), T(pb.v0)
    fwd_stats = []
    for _ in range(3):
        q, lam, fs = pkg.forward_step(scene, contacts, q_prev, v_prev, None, tuple(sc.gravity), eps=sc.eps)
        fwd_stats.append(fs)
        v_prev = (q - q_prev) / sc.h
        q_prev, q = q, None
    q_prev_adj = q_prev - v_prev * sc.h   # the differentiated step maps q_prev_adj -> q_adj
    q_adj = q_prev
    lam_adj = lam.contiguous()
    # centroid loss L = ||mean(q) - c_tgt||^2, target 1 mm further down the slope
    c_tgt = q_adj.mean(0) + 1e-3 * T(sc.planes[0].t1)
    dL_dq = (2.0 * (q_adj.mean(0) - c_tgt) / sc.n_verts).expand(sc.n_verts, 3).contiguous()
    dL_dv = torch.zeros_like(dL_dq)
    outputs = {k: torch.empty(v, dtype=torch.float64, device=dev) for k, v in (
        ("dL_dq_prev", (sc.n_verts, 3)), ("dL_dv_prev", (sc.n_verts, 3)), ("dL_dfext", (sc.n_verts, 3)),
        ("z", (sc.n_verts, 3)), ("dL_dE", (sc.n_tets,)), ("dL_dnu", (sc.n_tets,)), ("dL_dmu", (1,)),
        ("dL_dmu_contact", (ct.n,)))}
    stream = torch.cuda.Stream(dev)
    flush = torch.empty(512 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)

    def one(mem="device", ins=None, outs=None, prec="fp64", cap="fp64", bindings=None):
        a = ins or (q_adj, q_prev_adj, lam_adj, dL_dq, dL_dv, contacts)
        return pkg.adjoint_step(scene, a[5], a[0], a[1], a[2], a[3], a[4], eps=sc.eps, rtol=1e-8, memory=mem,
                                outputs=outs or outputs, stream=stream.cuda_stream, precision=prec,
                                cap_precision=cap, bindings=bindings)

    variants = {"fp64": ("fp64", "fp64"), "mixed": ("mixed", "mixed"), "mixed_cap64": ("mixed", "fp64")}
    # accuracy of the mixed variants against plain FP64 on the same inputs
    ref = {k: v.clone() for k, v in one(prec="fp64")[0].items()}
    errs = {}
    grads_by = {"fp64": ref}  # kept for the oracle comparison of the CPU-baseline leg
    for name, (pr, cp) in variants.items():
        if name == "fp64":
            continue
        g_ = one(prec=pr, cap=cp)[0]
        grads_by[name] = {k: v.clone() for k, v in g_.items()}
        errs[name] = max(float((torch.linalg.norm(g_[k] - ref[k]) / torch.linalg.norm(ref[k]).clamp_min(1e-300)).item())
                         for k in ref)
    torch.cuda.synchronize(dev)

    def timed(pr, cp, steps, **kw):
        with torch.cuda.stream(stream):
            for _ in range(args.warmup):
                one(prec=pr, cap=cp, **kw)
        torch.cuda.synchronize(dev)
        if world > 1:
            dist.barrier()
        ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for _ in range(steps)]
        sts = []
        with torch.cuda.stream(stream):
            for i in range(steps):
                flush.zero_()  # evict the previous step's working set from L2
                ev[i][0].record(stream)
                _, st = one(prec=pr, cap=cp, **kw)
                ev[i][1].record(stream)
                sts.append(st)
        torch.cuda.synchronize(dev)
        tot = sum(x.elapsed_time(y) for x, y in ev)
        if world > 1:
            t = torch.tensor([tot], device=dev)
            dist.all_reduce(t, op=dist.ReduceOp.MAX)
            tot = float(t.item())
        return tot, sts

    # the headline variant: the fastest mixed variant within 1e-3 of plain FP64, else plain FP64
    head = "mixed" if errs["mixed"] <= 1e-3 else ("mixed_cap64" if errs["mixed_cap64"] <= 1e-3 else "fp64")
    results = {}
    for name in ("fp64", "mixed_cap64", "mixed"):
        if name == head:
            continue
        results[name] = timed(*variants[name], max(3, args.steps // 2))
    clocks = ClockSampler(local)
    clocks.start()
    t_wall0 = time.perf_counter()
    torch.cuda.nvtx.range_push("timed")
    total_ms, stats = timed(*variants[head], args.steps)
    torch.cuda.nvtx.range_pop()
    t_wall = time.perf_counter() - t_wall0
    clk = clocks.stop()
    results[head] = (total_ms, stats)
    value = world * args.steps / (total_ms / 1e3)
    rate = {k: world * len(v[1]) / (v[0] / 1e3) for k, v in results.items()}

    # ---- end to end through the C-ABI with host buffers (copies inside the timed region) ----
    pin = lambda t: t.cpu().pin_memory()  # noqa: E731
    h_contacts = pkg.Contacts(pin(contacts.vertex), pin(contacts.frame), pin(contacts.d_n), pin(contacts.mu), None,
                              pin(contacts.region), contacts.n_regions)
    h_in = (pin(q_adj), pin(q_prev_adj), pin(lam_adj), pin(dL_dq), pin(dL_dv), h_contacts)
    h_out = {k: torch.empty(v.shape, dtype=torch.float64).pin_memory() for k, v in outputs.items()}
    h2d = sum(t.numel() * t.element_size() for t in h_in[:5]) + sum(
        t.numel() * t.element_size() for t in (h_contacts.vertex, h_contacts.frame, h_contacts.d_n, h_contacts.mu,
                                                h_contacts.region))
    d2h = sum(t.numel() * t.element_size() for t in h_out.values())
    with torch.cuda.stream(stream):
        e2e_t = []
        if not args.no_e2e:
            one("host", h_in, h_out, *variants[head])
        for _ in range(0 if args.no_e2e else max(3, args.steps // 2)):
            flush.zero_()
            torch.cuda.synchronize(dev)
            t0 = time.perf_counter()
            one("host", h_in, h_out, *variants[head])  # synchronous: returns once outputs are in host memory
            e2e_t.append(time.perf_counter() - t0)
    e2e_value = world / (sum(e2e_t) / len(e2e_t)) if e2e_t else None

    # ---- roofline of the dominant kernel ----
    # The Krylov loop dominates the step, and in it the product with A^{-1} = P^T S^T S P (two
    # launches of k_spmv_chunks, S then S^T, with 3 right-hand sides): it is timed live here through
    # ncpadj_elastic_solve on its own stream (the same kernels on the same data, FP64 values).
    it = statistics.median(s["iterations"] for s in stats)
    ncap = stats[0]["capacitance_dim"]
    info = scene.info()
    hbm_peak, hbm_src = peaks()
    launches = int(statistics.median(s["kernel_launches"] for s in stats))
    n3 = 3 * sc.n_verts
    roof = apply_roofline(pkg, torch, dev, scene, 50)
    roof["note"] = ("burst figure: applies replayed back to back from a captured graph, S and S^T "
                    "(53 MB on the beam) L2-resident between launches")

    # ---- the other constitutive models (App. B.2) and stiff bindings, same scene and state ----
    # (one rank only: a failure here must not leave other ranks waiting in a collective)
    models_res = None
    if world == 1 and not args.no_models:
        models_res = models_leg(pkg, torch, dev, scene, sc.n_verts, q_adj,
                                lambda **kw: timed(*variants[head], max(3, args.steps // 4), **kw))

    # ---- the batched workload ----
    batch_res = None
    if not args.no_batch:
        try:
            batch_res = batched(pkg, torch, dev, max(3, args.steps // 4), 1)
        except Exception as e:  # noqa: BLE001
            batch_res = {"error": str(e)[:300]}

    sphere_res = None
    if args.sphere:
        try:
            sphere_res = sphere(pkg, torch, dev, max(3, args.steps // 4), 1)
        except Exception as e:  # noqa: BLE001
            sphere_res = {"error": str(e)[:300]}

    quad_res = None
    if args.quadruped:
        try:
            quad_res = quadruped_measure(pkg, torch, dev, max(2, args.steps // 4), 1, args.quad_scale)
        except Exception as e:  # noqa: BLE001
            quad_res = {"error": str(e)[:300]}

    # ---- CPU baseline: the oracle, one thread, bounded sample ----
    # The oracle runs at the bench's own state (the GPU forward's), on the same seeds, so the same
    # runs also give each GPU variant's gradient error against the oracle.
    cpu, err_oracle = None, None
    if rank == 0 and not args.no_cpu_baseline:
        arrays = {"q": q_adj.cpu().numpy(), "q_prev": q_prev_adj.cpu().numpy(), "dL_dq": dL_dq.cpu().numpy(),
                  "dL_dv": dL_dv.cpu().numpy()}
        for vname, gv in grads_by.items():
            for k, v in gv.items():
                arrays[f"{vname}/{k}"] = v.cpu().numpy()
        cpu, err_oracle = cpu_baseline_leg(arrays)
    if rank == 0:
        print(json.dumps({
            "metric": METRIC, "value": value, "unit": "gradients/s", "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": total_ms / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64" if head == "fp64" else "f32+f64",
            "data": "synthetic",
            "config": {"workload": WORKLOAD, "variant": head,
                       "precision": {"fp64": "plain FP64", "mixed": "FP32 matrix/preconditioner/capacitance factor, FP64 "
                                     "Krylov reductions", "mixed_cap64": "FP32 matrix/preconditioner, FP64 capacitance "
                                     "factor and Krylov reductions"}[head],
                       "gradients_per_s": rate, "max_rel_err_vs_fp64": errs, "max_rel_err_vs_oracle": err_oracle,
                       "preconditioner": "Woodbury",
                       "solver": "GMRES(64)", "rtol": 1e-8, "krylov_iterations": it, "capacitance_dim": ncap,
                       "l2": "flushed (512 MB write) before every timed step", "parallelism": f"replicas x{world}",
                       "wall_s": t_wall, "stage_ms": {k: statistics.mean(s[k] for s in stats) for k in
                                                      ("ms_assemble", "ms_setup", "ms_krylov", "ms_contract",
                                                       "ms_cap_inverse")},
                       "forward_newton_iters": [f["newton_iters"] for f in fwd_stats],
                       "forward_residual": [f["residual"] for f in fwd_stats],
                       "nnz_L": info["nnz_L"], "nnz_Linv": info["nnz_Linv"], "batched": batch_res,
                       **({"models": models_res} if models_res is not None else {}),
                       **({"sphere": sphere_res} if sphere_res is not None else {}),
                       **({"quadruped": quad_res} if quad_res is not None else {})},
            "roofline": roof, "cpu_baseline": cpu,
            "e2e": {"value": e2e_value, "unit": "gradients/s", "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h},
            "gpu_launches": launches * args.steps, "clocks": clk,
        }))
    if world > 1:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
