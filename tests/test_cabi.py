"""The C ABI library loads and exports every entry point include/dgs.h declares (CPU)."""
import os
import re

from paper_2606_17212_b300 import build, dgs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared():
    src = open(os.path.join(ROOT, "include", "dgs.h")).read()
    return sorted(set(re.findall(r"DGS_API\s+[\w\s\*]+?\b(dgs_\w+)\s*\(", src)))


def test_header_declares_the_binding_exports():
    assert sorted(dgs.EXPORTS) == declared()


def test_library_loads_and_exports_every_symbol():
    build.build()
    L = dgs.lib()
    for name in declared():
        assert hasattr(L, name), name
    assert L.dgs_version() == 1


def test_library_binds_every_symbol_at_load():
    """Loading with immediate binding fails if any symbol of the library is left
    undefined (e.g. a launcher declared with one signature and defined with another)."""
    import ctypes
    import os
    from paper_2606_17212_b300 import dgs
    ctypes.CDLL(dgs.LIB_PATH, mode=os.RTLD_NOW | os.RTLD_LOCAL)
