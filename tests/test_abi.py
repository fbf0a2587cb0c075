"""CPU-only checks of the C ABI boundary: the library loads and exports every
entry point that include/tm.h declares, and the Python binding marshals each
one (no compute calls; no GPU needed)."""
import ctypes
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def header_functions():
    names = []
    for fn in sorted(os.listdir(os.path.join(ROOT, "include"))):
        if fn.endswith(".h"):
            text = open(os.path.join(ROOT, "include", fn)).read()
            text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
            names += re.findall(r"^\s*(?:const\s+)?[A-Za-z_][A-Za-z0-9_]*\s*\*?\s*(tm_[a-z0-9_]+)\s*\(", text, re.M)
    return sorted(set(names))


@pytest.fixture(scope="module")
def built():
    from paper_2310_02800_gb300 import build
    return build.build()


def test_header_declares_the_boundary():
    names = header_functions()
    for required in ("tm_graph_load", "tm_graph_free", "tm_query_compile", "tm_count", "tm_enumerate",
                     "tm_count_batch", "tm_serve_start", "tm_serve_submit", "tm_serve_poll", "tm_result_release",
                     "tm_serve_stop", "tm_status_str"):
        assert required in names


def test_library_exports_every_declared_symbol(built):
    lib = ctypes.CDLL(built)
    missing = [n for n in header_functions() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_covers_every_symbol(built):
    import paper_2310_02800_gb300 as tmg
    bound = {name for name, _, _ in tmg._SIGS}
    assert set(header_functions()) <= bound
    L = tmg.lib()
    assert L.tm_status_str(0) == b"ok"
    assert b"truncated" in L.tm_status_str(3)


def test_struct_layouts_match_header():
    """Sizes of the ABI structs as the binding sees them (C layout rules)."""
    import paper_2310_02800_gb300 as tmg
    assert ctypes.sizeof(tmg._Edges) == 8 * 2 + 8 * 5 + 8
    assert ctypes.sizeof(tmg._Motif) == 4 + 4 + 8 + 8 + 8 + 7 * 8 + 16 + 16 + 4 + 4 * 3 + 4 * 8
    assert ctypes.sizeof(tmg.Tuning) == 16
    assert ctypes.sizeof(tmg._Work) == 8 * (1 + 8 + 8 + 1 + 1)
    assert ctypes.sizeof(tmg._ServeCfg) == 8 + 4 * 4 + 8 + 8


def test_missing_library_fails_loudly(tmp_path, monkeypatch):
    import paper_2310_02800_gb300 as tmg
    monkeypatch.setattr(tmg, "_SO", str(tmp_path / "absent.so"))
    monkeypatch.setattr(tmg, "_lib", None)
    with pytest.raises(ImportError):
        tmg.lib()
