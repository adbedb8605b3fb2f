"""The C-ABI library loads and exports every entry point the header declares (CPU only)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for f in os.listdir(os.path.join(ROOT, "include")):
        if f.endswith(".h"):
            src = open(os.path.join(ROOT, "include", f)).read()
            src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
            names |= set(re.findall(r"\b(ncpadj_[a-z_]+)\s*\(", src))
    return sorted(names)


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__ as g
    g.build()
    from paper_2603_16478_gb300 import load_library
    return load_library()


def test_header_declares_entry_points():
    names = _declared()
    assert "ncpadj_adjoint_step" in names and "ncpadj_scene_create" in names


def test_library_exports_every_declared_symbol(lib):
    for name in _declared():
        assert hasattr(lib, name), name


def test_version_and_status_strings(lib):
    assert b"sm_103a" in lib.ncpadj_version()
    assert lib.ncpadj_status_string(0) == b"OK"
    assert lib.ncpadj_status_string(5) == b"NOT_CONVERGED"


def test_null_arguments_are_rejected_without_a_gpu(lib):
    # INVALID_ARG before anything touches the device
    assert lib.ncpadj_ctx_create(0, None) == 1
    assert lib.ncpadj_scene_get_info(None, None) == 1
    assert lib.ncpadj_adjoint_step(None, None, None, None, None, None, None, None, None) != 0
    assert len(lib.ncpadj_last_error()) > 0


def test_binding_fails_loudly_without_library(tmp_path):
    from paper_2603_16478_gb300 import binding
    with pytest.raises(RuntimeError, match="missing"):
        binding.load_library(str(tmp_path / "nope.so"))


def test_ctypes_structs_match_the_header(tmp_path):
    """Every struct the binding mirrors has the header's size and field offsets (compiled by gcc)."""
    import shutil
    import subprocess
    from paper_2603_16478_gb300 import binding as B
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pairs = {"ncpadj_scene_desc": B._SceneDesc, "ncpadj_shell_desc": B._ShellDesc,
             "ncpadj_scene_info": B._SceneInfo, "ncpadj_contacts": B._Contacts,
             "ncpadj_bindings": B._Bindings, "ncpadj_state": B._State, "ncpadj_seed": B._Seed,
             "ncpadj_grads": B._Grads, "ncpadj_options": B._Options, "ncpadj_stats": B._Stats,
             "ncpadj_forward_input": B._ForwardInput, "ncpadj_forward_stats": B._ForwardStats}
    # the ctypes field names follow the header's, except lambda (a Python keyword)
    rename = {("ncpadj_state", "lam"): "lambda"}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "ncpadj.h"', "int main(void) {"]
    for cname, py in pairs.items():
        lines.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f, _ in py._fields_:
            cf = rename.get((cname, f), f)
            lines.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {cf}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = dict(line.rsplit(" ", 1) for line in subprocess.run([str(exe)], check=True, capture_output=True,
                                                               text=True).stdout.splitlines())
    for cname, py in pairs.items():
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f, _ in py._fields_:
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)


def test_plain_c_client_links_and_runs(lib, tmp_path):
    """A C program (tests/c_client.c) built with gcc against the header and the library calls the
    entry points that need no device."""
    import shutil
    import subprocess
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    libdir = os.path.join(ROOT, "paper_2603_16478_gb300")
    exe = tmp_path / "c_client"
    subprocess.run([cc, "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"),
                    os.path.join(ROOT, "tests", "c_client.c"), "-L", libdir, "-lncpadj",
                    "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    r = subprocess.run([str(exe)], capture_output=True, text=True)
    assert r.returncode == 0 and r.stdout.strip().endswith("PASS"), r.stdout + r.stderr
