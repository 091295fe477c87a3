"""The C-ABI library loads and exports every function include/sg.h declares
(no compute calls: runs without a GPU)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    src = open(os.path.join(ROOT, "include", "sg.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(sg_[a-z_0-9]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for n in ["sg_ctx_create", "sg_add_transmon", "sg_add_fluxonium", "sg_add_coupling",
              "sg_add_drive", "sg_prepare", "sg_evolve", "sg_fidelity", "sg_fidelity_grad",
              "sg_server_create", "sg_server_submit", "sg_server_poll"]:
        assert n in names


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2406_18155_gb300 import build, capi
    try:
        build.build()
    except RuntimeError as e:          # no nvcc on this machine
        pytest.skip(str(e))
    lib = ctypes.CDLL(capi.LIB_PATH)
    for n in declared_functions():
        assert hasattr(lib, n), n
    # the binding mirrors the header one to one
    assert set(capi.SIGNATURES) == set(declared_functions())
    assert capi.lib().sg_version().decode().startswith("supergpu")


def test_binding_fails_loudly_without_the_library(monkeypatch, tmp_path):
    from paper_2406_18155_gb300 import capi
    monkeypatch.setattr(capi, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(capi, "_lib", None)
    with pytest.raises(RuntimeError, match="no CPU path"):
        capi.lib()


def test_binding_structs_match_the_header_layout(tmp_path):
    """Every ctypes struct of the binding has the C header's size and field offsets
    (a small C program compiled with the host compiler prints them)."""
    import shutil
    import subprocess
    from paper_2406_18155_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    structs = [capi.sg_pulse, capi.sg_evolve_opts, capi.sg_request, capi.sg_result, capi.sg_stats]
    lines = ['#include <stdio.h>', '#include <stddef.h>', '#include "sg.h"', "int main(void) {"]
    for st in structs:
        name = st.__name__
        lines.append(f'  printf("{name} size %zu\\n", sizeof({name}));')
        for f in st._fields_:
            lines.append(f'  printf("{name} {f[0]} %zu\\n", offsetof({name}, {f[0]}));')
    lines += ["  return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st in structs:
        name = st.__name__
        assert got[(name, "size")] == ctypes.sizeof(st), name
        for f in st._fields_:
            assert got[(name, f[0])] == getattr(st, f[0]).offset, (name, f[0])


def test_binding_constants_match_the_header(tmp_path):
    """Every SG_* constant of the binding has the header's value (status codes,
    solvers, compensation, basis, operators, envelopes, precisions, frames, kinds)."""
    import shutil
    import subprocess
    from paper_2406_18155_gb300 import capi
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    names = sorted(n for n in dir(capi) if re.fullmatch(r"SG_[A-Z0-9_]+", n) and isinstance(getattr(capi, n), int))
    assert len(names) > 20
    lines = ['#include <stdio.h>', '#include "sg.h"', "int main(void) {"]
    lines += [f'  printf("{n} %d\\n", (int)({n}));' for n in names]
    lines += ["  return 0;", "}"]
    src = tmp_path / "consts.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "consts"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {l.split()[0]: int(l.split()[1]) for l in out if l.strip()}
    for n in names:
        assert got[n] == getattr(capi, n), n
