"""The C-ABI library builds, loads and exports every entry point that
include/*.h declares (no GPU needed, no compute calls)."""
import ctypes
import glob
import os
import re
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared_functions():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"^\s*(?:const\s+)?[A-Za-z_][\w\s\*]*?\b([a-z_][a-z0-9_]*)\s*\(", text, flags=re.M):
            name = m.group(1)
            if name not in ("if", "while", "for", "return", "sizeof"):
                names.add(name)
    return names


@pytest.fixture(scope="module")
def libpath():
    from paper_2605_05469_gb300 import LIB_PATH, build
    if not os.path.exists(LIB_PATH):
        build.build()
    return LIB_PATH


def test_header_declares_the_boundary():
    names = _declared_functions()
    for required in ("pic_create", "pic_init", "pic_deposit", "poisson_solve", "poisson_solve_ex",
                     "pic_gather_push", "pic_field_energy", "pic_destroy", "pic_strerror"):
        assert required in names


def test_library_exports_every_declared_symbol(libpath):
    out = subprocess.run(["nm", "-D", "--defined-only", libpath], capture_output=True, text=True, check=True).stdout
    exported = {line.split()[-1] for line in out.splitlines() if " T " in line}
    missing = _declared_functions() - exported
    assert not missing, f"declared in include/*.h but not exported: {sorted(missing)}"


def test_library_loads_and_binding_resolves(libpath):
    ctypes.CDLL(libpath)
    import paper_2605_05469_gb300 as pg
    L = pg.lib()
    for name in pg.exported_symbols():
        assert hasattr(L, name)
    assert pg.strerror(pg.PIC_ENOCONV).startswith("solver did not converge")
