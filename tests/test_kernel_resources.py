"""Register spills of the CUDA kernels, from the compiler's resource report (CPU only: nvcc
cross-compiles for sm_103a with the library's own flags and -Xptxas -v).  No kernel may spill,
except the two wide Gauss-Jordan variants for FP32 capacitance blocks above 4,096 rows, whose
register panels of 64 values are known to exceed the budget."""
import os
import re
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

import pytest

from paper_2603_16478_gb300 import build as B

SOURCES = ("elem.cu", "linalg.cu", "gj.cu", "bgj.cu")
# k_gj_cols<float, 4, 16, false> and k_gj_cols<float, 2, 32, false> (mangled template arguments)
ALLOWED = (re.compile(r"k_gj_colsIfLi4ELi16ELb0E"), re.compile(r"k_gj_colsIfLi2ELi32ELb0E"))


def _report(src, tmp):
    nvcc = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    r = subprocess.run([nvcc, *B.ARCH, *B.FLAGS, "-Xptxas", "-v", "-c", os.path.join(B.CSRC, src),
                        "-o", os.path.join(tmp, src + ".o")], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr[-2000:]
    return r.stderr


def test_no_kernel_spills_registers(tmp_path):
    if shutil.which("nvcc") is None and not os.path.exists("/usr/local/cuda/bin/nvcc"):
        pytest.skip("needs nvcc")
    with ThreadPoolExecutor(len(SOURCES)) as ex:
        reports = list(ex.map(lambda s: _report(s, str(tmp_path)), SOURCES))
    kernels, spills = 0, []
    for text in reports:
        name = None
        for line in text.splitlines():
            m = re.search(r"Compiling entry function '([^']+)'", line)
            if m:
                name = m.group(1)
                kernels += 1
                continue
            m = re.search(r"(\d+) bytes spill stores, (\d+) bytes spill loads", line)
            if m and name and (int(m.group(1)) or int(m.group(2))):
                if not any(p.search(name) for p in ALLOWED):
                    spills.append((name, line.strip()))
    assert kernels > 40  # the report was read
    assert not spills, spills
