"""CPU checks of the C ABI: the library builds, loads and exports every symbol of include/vie.h."""
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "vie.h")).read()
    return sorted(set(re.findall(r"\b(vie_[a-z_]+)\s*\(", src)))


def test_header_declares_python_exports():
    import paper_2111_01730_gb300 as pkg

    assert sorted(pkg.EXPORTS) == _declared()


def test_library_loads_and_exports_all_symbols():
    import paper_2111_01730_gb300 as pkg

    if not os.path.exists(pkg.LIB_PATH):
        from paper_2111_01730_gb300 import build_lib

        build_lib.build()
    lib = pkg.load_library()
    for name in _declared():
        assert hasattr(lib, name), name
