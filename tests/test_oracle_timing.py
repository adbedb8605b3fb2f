"""The oracle timing harness behind the bench's CPU baseline (CPU only): at a given state it times
the oracle adjoint and reports the relative error of stored gradients against it."""
import json
import os
import subprocess
import sys

import numpy as np

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def test_state_mode_reports_the_planted_errors(tmp_path):
    from oracle.timing import KEYS, beam_case
    st, s, q_prev, dq, dv = beam_case()
    ref = st.adjoint(s, q_prev, dq, dv)
    arrays = {"q": s.q, "q_prev": q_prev, "dL_dq": dq, "dL_dv": dv}
    for key, ok in KEYS:
        r = np.asarray(ref[ok])
        arrays["exact/" + key] = r
        arrays["off/" + key] = r * (1.0 + (1e-3 if key == "dL_dE" else 0.0))
    path = str(tmp_path / "state.npz")
    np.savez(path, **arrays)
    out = subprocess.run([sys.executable, "-m", "oracle.timing", "--steps", "1", "--warmup", "0", "--state", path],
                         cwd=ROOT, capture_output=True, text=True, timeout=600)
    assert out.returncode == 0, out.stderr[-2000:]
    d = json.loads(out.stdout.strip().splitlines()[-1])
    assert d["state"] == "given" and len(d["seconds"]) == 1 and d["n_contacts"] == 451
    assert d["rel_err_vs_oracle"]["exact"] < 1e-12
    assert abs(d["rel_err_vs_oracle"]["off"] - 1e-3) < 1e-9
