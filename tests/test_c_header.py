"""include/hzs.h is a C header: a C99 translation unit that includes it and takes the
address of every declared entry point compiles warning-free with gcc and links
against libhzs.so (no GPU needed; the program is built, not run); and the Python
binding's ctypes structures have the header's struct sizes and field offsets."""
import ctypes
import os
import re
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "hzs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(hzs_[a-z_0-9]+)\s*\(", src)))


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_header_is_c99_and_links(tmp_path):
    from paper_2408_03571_gb300 import build
    lib = build.build()
    names = _declared()
    c = tmp_path / "uses_hzs.c"
    c.write_text(
        "#include <stdio.h>\n#include \"hzs.h\"\n"
        "int main(void) {\n"
        "    hzs_grid_desc gd = {65, HZS_DIRICHLET, 20.0, NULL, 4, 2, 0};\n"
        "    hzs_precond_desc pd = {HZS_SHS2, HZS_COARSE_B2, 8, HZS_MIXED, 1, HZS_COARSE_SOLVER_AUTO, 0,\n"
        "                           HZS_SCALING_OWNER, 0, 0, 0};\n"
        "    hzs_solve_desc sd = {1e-7, 200, HZS_SOLVE_GRAPH};\n"
        "    hzs_solve_info info; hzs_precond_info pinfo; hzs_pipe_rates rates;\n"
        "    void (*fns[])(void) = {\n"
        + "".join(f"        (void (*)(void))&{n},\n" for n in names)
        + "    };\n"
        "    (void)gd; (void)pd; (void)sd; (void)info; (void)pinfo; (void)rates;\n"
        "    printf(\"%u %s\\n\", (unsigned)(sizeof fns / sizeof fns[0]), hzs_status_string(HZS_OK));\n"
        "    return 0;\n}\n")
    exe = tmp_path / "uses_hzs"
    libdir = os.path.dirname(lib)
    cmd = ["gcc", "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
           str(c), "-o", str(exe), "-L", libdir, "-lhzs", "-Wl,--unresolved-symbols=ignore-in-shared-libs"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


STRUCTS = {
    "hzs_grid_desc": "GridDesc",
    "hzs_precond_desc": "PrecondDesc",
    "hzs_solve_desc": "SolveDesc",
    "hzs_solve_info": "SolveInfo",
    "hzs_precond_info": "PrecondInfo",
    "hzs_pipe_rates": "PipeRates",
}


@pytest.mark.skipif(shutil.which("gcc") is None, reason="needs gcc")
def test_binding_structs_match_the_header(tmp_path):
    """The ctypes structures of the Python binding have the C structs' size and field
    offsets (a mismatch would pass wrong arguments without any error)."""
    from paper_2408_03571_gb300 import hzs
    lines = ["#include <stdio.h>", "#include <stddef.h>", "#include \"hzs.h\"", "int main(void) {"]
    for cname, pyname in STRUCTS.items():
        lines.append(f'    printf("{cname} size %zu\\n", sizeof({cname}));')
        for field, _ in getattr(hzs, pyname)._fields_:
            lines.append(f'    printf("{cname} {field} %zu\\n", offsetof({cname}, {field}));')
    lines += ["    return 0;", "}"]
    c = tmp_path / "layout.c"
    c.write_text("\n".join(lines) + "\n")
    exe = tmp_path / "layout"
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(c), "-o",
                        str(exe)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.split("\n")
    c_layout = {}
    for ln in out:
        if ln:
            s, f, v = ln.split()
            c_layout[(s, f)] = int(v)
    for cname, pyname in STRUCTS.items():
        cls = getattr(hzs, pyname)
        assert c_layout[(cname, "size")] == ctypes.sizeof(cls), cname
        for field, _ in cls._fields_:
            assert c_layout[(cname, field)] == getattr(cls, field).offset, (cname, field)
