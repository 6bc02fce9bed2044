"""The C-ABI library builds, loads without a GPU and exports every symbol
that include/*.h declares. No compute call is made here."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

from paper_2509_19703_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(h).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[\w\s\*]+?\b(gumap_\w+)\s*\(", text, flags=re.M):
            names.add(m.group(1))
    return sorted(names)


@pytest.fixture(scope="module")
def lib_path():
    return _build.build()


def test_header_declares_entry_points():
    names = declared_symbols()
    for must in ("gumap_knn_create", "gumap_knn_run", "gumap_knn_destroy", "gumap_status_string"):
        assert must in names, names


def test_library_exports_every_declared_symbol(lib_path):
    out = subprocess.run(["nm", "-D", "--defined-only", lib_path], capture_output=True, text=True, check=True).stdout
    exported = set(re.findall(r"\bT (gumap_\w+)", out))
    missing = [s for s in declared_symbols() if s not in exported]
    assert not missing, f"declared but not exported: {missing}"


def declared_arities():
    """Entry point -> number of parameters, from the declarations of include/*.h."""
    out = {}
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = re.sub(r"/\*.*?\*/", "", open(h).read(), flags=re.S)
        for m in re.finditer(r"\b(gumap_\w+)\s*\(([^;{()]*)\)\s*;", text):
            params = m.group(2).strip()
            out[m.group(1)] = 0 if params in ("", "void") else len(params.split(","))
    return out


def test_binding_matches_the_header():
    """The ctypes binding knows every declared entry point, with as many
    arguments as the header declares (no load, no GPU)."""
    from paper_2509_19703_gb300 import gumap

    sigs = gumap._signatures()
    decl = declared_arities()
    assert set(decl) == set(sigs), (sorted(set(decl) - set(sigs)), sorted(set(sigs) - set(decl)))
    wrong = {name: (n, len(sigs[name][0])) for name, n in decl.items() if len(sigs[name][0]) != n}
    assert not wrong, wrong


STRUCTS = {"_Stats": "gumap_knn_stats", "_Info": "gumap_knn_info", "_Tune": "gumap_tune_result",
           "_ServerOpts": "gumap_server_opts", "_Result": "gumap_result", "_ServerStats": "gumap_server_stats",
           "_SpectralInfo": "gumap_spectral_info"}


def test_binding_structs_match_the_header(tmp_path):
    """Every ctypes structure of the binding has the size and field offsets
    of its C struct, as gcc lays it out from include/gumap.h."""
    from paper_2509_19703_gb300 import gumap

    lines = ['#include <stddef.h>', '#include <stdio.h>', '#include "gumap.h"', "int main(void) {"]
    for py, c in STRUCTS.items():
        lines.append(f'printf("{py} size %zu\\n", sizeof({c}));')
        for field, _ in getattr(gumap, py)._fields_:
            lines.append(f'printf("{py} {field} %zu\\n", offsetof({c}, {field}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "layout.c"
    src.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c11", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        py, what, val = line.split()
        got[(py, what)] = int(val)
    for py in STRUCTS:
        cls = getattr(gumap, py)
        assert got[(py, "size")] == ctypes.sizeof(cls), py
        for field, _ in cls._fields_:
            assert got[(py, field)] == getattr(cls, field).offset, (py, field)


def test_library_loads_and_answers_host_only_calls(lib_path):
    lib = ctypes.CDLL(lib_path)
    lib.gumap_status_string.restype = ctypes.c_char_p
    assert lib.gumap_status_string(0) == b"GUMAP_OK"
    assert lib.gumap_status_string(7) == b"GUMAP_ERR_TIMEOUT"
    lib.gumap_last_error.restype = ctypes.c_char_p
    assert isinstance(lib.gumap_last_error(), bytes)


def test_binding_argument_checks_without_gpu(lib_path):
    """Invalid arguments are rejected on the host before any device work."""
    from paper_2509_19703_gb300 import gumap
    import numpy as np
    rp = np.array([0, 1, 2], dtype=np.int32)
    col = np.array([1, 0], dtype=np.int32)
    with pytest.raises(gumap.GumapError) as e:
        gumap.gumap_knn_create(rp, col, 2, 2, k=5)  # k > n - 1
    assert e.value.status == gumap.ERR_INVALID_ARG
    with pytest.raises(gumap.GumapError) as e:
        gumap.gumap_knn_create(rp, col, 2, 2, k=1, mode=7)
    assert e.value.status == gumap.ERR_INVALID_ARG


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_2509_19703_gb300 import gumap
    monkeypatch.setattr(gumap, "_lib", None)
    monkeypatch.setattr(gumap._build, "LIB", str(tmp_path / "absent.so"))
    with pytest.raises(RuntimeError, match="no CPU fallback"):
        gumap.load()


def test_binding_constants_match_the_header():
    """Every GUMAP_* integer constant of the header that the binding also
    defines (without the prefix) has the same value there."""
    import re

    from paper_2509_19703_gb300 import gumap
    text = open(os.path.join(ROOT, "include", "gumap.h")).read()
    pairs = re.findall(r"^#define\s+GUMAP_(\w+)\s+(0x[0-9A-Fa-f]+|-?\d+)\b", text, flags=re.M)
    assert len(pairs) > 20
    checked = 0
    for name, val in pairs:
        if hasattr(gumap, name):
            assert getattr(gumap, name) == int(val, 0), name
            checked += 1
    assert checked >= 20
