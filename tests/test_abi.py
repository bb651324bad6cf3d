"""The C ABI library loads and exports every symbol include/hpmc.h declares
(no GPU needed: no compute calls)."""
import ctypes
import os
import re

from paper_1509_04692_gb300 import build

HEADER = os.path.join(os.path.dirname(os.path.dirname(__file__)), "include", "hpmc.h")


def declared():
    txt = open(HEADER).read()
    return sorted(set(re.findall(r"^(?:int|const char\*)\s+(hpmc_\w+)\s*\(", txt, re.M)))


def test_library_builds_and_exports_every_declared_symbol():
    path = build.build()
    lib = ctypes.CDLL(path)
    names = declared()
    assert len(names) >= 19
    for n in names:
        assert hasattr(lib, n), n


def test_binding_lists_match_header():
    from paper_1509_04692_gb300 import hpmc
    assert sorted(hpmc.EXPORTS) == declared()


def test_strerror_without_gpu():
    from paper_1509_04692_gb300 import hpmc
    lib = hpmc.lib()
    assert lib.hpmc_strerror(-7).decode().startswith("a cell stencil")
    assert lib.hpmc_strerror(0).decode() == "ok"
