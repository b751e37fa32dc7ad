"""The C-ABI library builds for sm_103a, loads, and exports every symbol that
include/hba.h declares (no compute calls: no GPU needed)."""
from __future__ import annotations

import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    txt = open(os.path.join(ROOT, "include", "hba.h")).read()
    txt = re.sub(r"/\*.*?\*/", "", txt, flags=re.S)
    return sorted(set(re.findall(r"\b(hba_[a-z_0-9]+)\s*\(", txt)))


def test_header_declares_the_boundary():
    names = _declared()
    for must in ("hba_create", "hba_alloc_batch", "hba_free_batch", "hba_stats", "hba_destroy",
                 "hba_export_state", "hba_multi_create", "hba_multi_step", "hba_step_host",
                 "hba_step_host_async"):
        assert must in names


def test_library_exports_every_declared_symbol():
    from paper_2405_07079_gb300 import _lib
    from paper_2405_07079_gb300.build import build_library

    path = build_library()
    lib = ctypes.CDLL(path)
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing
    assert set(_declared()) == set(_lib.SIGNATURES), "binding and header disagree"
    assert _lib.load().hba_version().startswith(b"hba")


def test_invalid_arguments_rejected_without_device_work():
    """Argument checks that return before any CUDA call."""
    from paper_2405_07079_gb300 import _lib

    lib = _lib.load()
    h = ctypes.c_void_p()
    assert lib.hba_create(1 << 20, 100, 0, ctypes.byref(h)) == 1      # min_block not a power of two
    assert lib.hba_create(1 << 20, 4, 0, ctypes.byref(h)) == 1        # min_block < 8
    assert lib.hba_create(100, 256, 0, ctypes.byref(h)) == 1          # arena smaller than one block
    assert lib.hba_create(1 << 20, 256, 7, ctypes.byref(h)) == 1      # unknown policy
    assert lib.hba_create(1 << 40, 8, 0, ctypes.byref(h)) == 1        # more than 2^29 - 1 granules
    assert lib.hba_destroy(None) == 1
    assert lib.hba_step(None, None, 0, None, None, 0, None, None) == 1
    assert lib.hba_step_host(None, None, 0, None, None, 0, None, None) == 1
    assert lib.hba_step_host_async(None, None, 0, None, None, 0, None, None) == 1


def test_product_path_has_no_cpu_fallback():
    """The package never imports the oracle, and loading without the built
    library raises instead of falling back."""
    import paper_2405_07079_gb300 as pkg
    from paper_2405_07079_gb300 import _lib

    pkg_dir = os.path.dirname(pkg.__file__)
    for fn in os.listdir(pkg_dir):
        if fn.endswith(".py"):
            src = open(os.path.join(pkg_dir, fn)).read()
            assert "import oracle" not in src and "from oracle" not in src, fn
    try:
        _lib._lib_saved = _lib._lib
        _lib._lib = None
        import pytest
        with pytest.raises(OSError):
            _lib.load(os.path.join(ROOT, "no_such_dir", "libhba.so"))
    finally:
        _lib._lib = _lib._lib_saved


def test_every_imported_name_resolves():
    """Every name the tests, the bench and the entry module import from the
    package exists (checked without a GPU)."""
    import ast
    import glob
    import importlib
    import os

    import paper_2405_07079_gb300 as P

    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    files = (glob.glob(os.path.join(root, "tests", "*.py")) + glob.glob(os.path.join(root, "paper_2405_07079_gb300", "*.py"))
             + [os.path.join(root, "bench.py"), os.path.join(root, "__graft_entry__.py")])
    missing = []
    for f in files:
        with open(f) as fh:
            tree = ast.parse(fh.read())
        for node in ast.walk(tree):
            if isinstance(node, ast.ImportFrom) and node.module in ("paper_2405_07079_gb300",
                                                                    "paper_2405_07079_gb300.hba"):
                mod = P if node.module == "paper_2405_07079_gb300" else importlib.import_module(node.module)
                for a in node.names:
                    sub = importlib.util.find_spec(f"paper_2405_07079_gb300.{a.name}")
                    if not hasattr(mod, a.name) and sub is None:
                        missing.append((os.path.basename(f), a.name))
    assert not missing, missing
