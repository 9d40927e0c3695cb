"""The C-ABI library loads and exports every entry point its header declares (CPU only)."""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for h in glob.glob(os.path.join(ROOT, "include", "*.h")):
        src = open(h).read()
        src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
        names |= set(re.findall(r"^(?:st_status|void|const char\s*\*)\s+(st_\w+)\s*\(", src, re.M))
    return names


@pytest.fixture(scope="module")
def lib():
    import __graft_entry__

    __graft_entry__.build()
    from paper_2603_26691_gb300 import _lib

    return _lib.load()


def test_header_declares_the_paper_calls():
    names = _declared()
    for n in ("st_create_grid", "st_set_fluid", "st_add_particles", "st_step", "st_get_sources", "st_reorder"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    for name in sorted(_declared()):
        assert hasattr(lib, name), name


def test_binding_covers_every_declared_symbol():
    from paper_2603_26691_gb300 import _lib

    assert _declared() == set(_lib.SIGNATURES)


def test_library_targets_sm_103a_only():
    from paper_2603_26691_gb300 import build

    assert build.ARCH == ["-gencode", "arch=compute_103a,code=sm_103a"]


def test_no_cpu_fallback_when_library_missing(monkeypatch, tmp_path):
    from paper_2603_26691_gb300 import _lib, build

    monkeypatch.setattr(build, "LIB", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    with pytest.raises(ImportError):
        _lib.load()
