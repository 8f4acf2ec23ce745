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
