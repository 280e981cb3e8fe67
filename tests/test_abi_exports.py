"""The C ABI library loads and exports every function include/tw.h declares
(no compute calls: this runs without a GPU)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if not fn.endswith(".h"):
            continue
        src = open(os.path.join(ROOT, "include", fn)).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b(tw_\w+)\s*\(", src, flags=re.M):
            names.append(m.group(1))
    return sorted(set(names))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ("tw_create", "tw_destroy", "tw_decide", "tw_decide_u32", "tw_solve", "tw_solve_batch",
                     "tw_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol():
    import __graft_entry__
    __graft_entry__.build()
    from paper_1709_09990_gb300 import native
    lib = ctypes.CDLL(native.LIB_PATH)
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_status_strings_without_gpu():
    from paper_1709_09990_gb300 import native
    assert native.strerror(0) == "ok"
    assert "memory cap" in native.strerror(2)
    assert native.lib().tw_abi_version() == 3


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    from paper_1709_09990_gb300 import native
    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "absent.so"))
    try:
        native.lib()
    except RuntimeError as e:
        assert "not built" in str(e)
    else:
        raise AssertionError("expected a loud failure")


def _struct_fields(src, name):
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    body = re.search(r"typedef struct \{([^{}]*)\}\s*" + name + r"\s*;", src).group(1)
    return re.findall(r"(\w+)\s*(?:\[[^\]]*\])?\s*;", body)


def test_binding_structs_match_the_header(tmp_path):
    # field names and order of the ctypes mirrors, and every offset and size
    # as gcc lays the header out on this machine
    import subprocess
    from paper_1709_09990_gb300 import native
    src = open(os.path.join(ROOT, "include", "tw.h")).read()
    probe = ["#include <stdio.h>", "#include <stddef.h>", '#include "tw.h"', "int main(void) {"]
    for cname, py in (("tw_config", native.Config), ("tw_stats", native.Stats)):
        fields = _struct_fields(src, cname)
        assert fields == [f[0] for f in py._fields_], cname
        probe.append(f'printf("{cname} %zu\\n", sizeof({cname}));')
        for f in fields:
            probe.append(f'printf("{cname}.{f} %zu\\n", offsetof({cname}, {f}));')
    probe.append("return 0; }")
    c = tmp_path / "probe.c"
    c.write_text("\n".join(probe))
    exe = tmp_path / "probe"
    subprocess.check_call(["gcc", "-I", os.path.join(ROOT, "include"), "-o", str(exe), str(c)])
    got = dict(line.split() for line in subprocess.check_output([str(exe)], text=True).splitlines())
    for cname, py in (("tw_config", native.Config), ("tw_stats", native.Stats)):
        assert int(got[cname]) == ctypes.sizeof(py), cname
        for f in _struct_fields(src, cname):
            assert int(got[f"{cname}.{f}"]) == getattr(py, f).offset, (cname, f)
