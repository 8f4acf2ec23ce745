"""The C-ABI library builds, loads and exports every entry point include/chfsi.h declares
(no compute calls: this runs without a GPU)."""
import os
import re

from paper_1305_5120_gb300 import chfsi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_functions():
    txt = open(os.path.join(ROOT, "include", "chfsi.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(chfsi_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = declared_functions()
    for required in ["chfsi_create", "chfsi_solve", "chfsi_next_in_sequence", "chfsi_destroy",
                     "chfsi_status_string", "chfsi_filter"]:
        assert required in names


def test_library_exports_every_declared_symbol():
    lib = chfsi.load()
    missing = [n for n in declared_functions() if not hasattr(lib, n)]
    assert not missing, missing
    # the binding wraps exactly the declared set
    assert sorted(chfsi.exported_names()) == declared_functions()


def test_status_strings_without_gpu():
    lib = chfsi.load()
    assert lib.chfsi_status_string(0) == b"ok"
    assert b"positive definite" in lib.chfsi_status_string(2)
    p = chfsi.default_params()
    assert (p.degree, p.degree_min, p.degree_max, p.max_iter, p.lanczos_steps) == (20, 10, 25, 50, 20)


def test_workspace_estimate_without_gpu():
    """chfsi_workspace_bytes is host arithmetic (the serving loop admits sequences by it):
    invalid sizes give 0; it grows with n and with the block; the mixed path needs more than
    the FP64 one; and it covers what a mixed solve must hold at once -- the four n x n FP64
    matrices (L, L^-1, H', the transform's temporary), the 12 BF16 digit planes of both
    operands of the n x n x n transform (12 * (n * 2n + 2n * 2n) * 2 bytes) and its split-K
    partial sums (one FP64 n x n product per 3584-term pass of the 2n real K terms)."""
    ws = chfsi.workspace_bytes
    fp64, mixed = chfsi.CHFSI_PREC_FP64, chfsi.CHFSI_PREC_MIXED
    assert ws(0, 10, 2) == 0 and ws(100, 0, 2) == 0 and ws(100, 10, -1) == 0
    for prec in (fp64, mixed):
        assert ws(1000, 100, 20, prec) <= ws(2000, 100, 20, prec) <= ws(4000, 100, 20, prec)
        assert ws(2000, 100, 20, prec) <= ws(2000, 200, 40, prec)
    for n, nev, nex in [(512, 32, 16), (2000, 200, 40), (13000, 1300, 260)]:
        k = nev + nex
        assert ws(n, nev, nex, mixed) > ws(n, nev, nex, fp64) >= 16 * (4 * n * n + 2 * n * k)
        passes = -(-2 * n // 3584)
        need = 16 * 4 * n * n + 2 * 12 * (n * 2 * n + 2 * n * 2 * n) + 16 * passes * n * n
        assert ws(n, nev, nex, mixed) >= need


def test_struct_layouts_match_the_header(tmp_path):
    """The binding's ctypes structures have the header's sizes and field offsets (a C probe
    compiled against include/chfsi.h prints them)."""
    import ctypes
    import shutil
    import subprocess
    import pytest
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    fields = {"chfsi_params": [f for f, _ in chfsi.Params._fields_],
              "chfsi_info": [f for f, _ in chfsi.Info._fields_]}
    lines = ["#include <stdio.h>", "#include <stddef.h>", '#include "chfsi.h"', "int main(void) {"]
    for st, fs in fields.items():
        lines.append(f'printf("{st} size %zu\\n", sizeof({st}));')
        for f in fs:
            lines.append(f'printf("{st} {f} %zu\\n", offsetof({st}, {f}));')
    lines += ["return 0;", "}"]
    src = tmp_path / "probe.c"
    src.write_text("\n".join(lines))
    exe = tmp_path / "probe"
    subprocess.run([cc, "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], check=True, capture_output=True, text=True).stdout.split("\n")
    got = {tuple(l.split()[:2]): int(l.split()[2]) for l in out if l.strip()}
    for st, cls in (("chfsi_params", chfsi.Params), ("chfsi_info", chfsi.Info)):
        assert got[(st, "size")] == ctypes.sizeof(cls), st
        for f, _ in cls._fields_:
            assert got[(st, f)] == getattr(cls, f).offset, (st, f)
