"""The C-ABI library builds for sm_103a, loads, and exports every function
declared in include/*.h (no compute calls: this runs without a GPU)."""
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
        for m in re.finditer(r"\b(?:int|void|const char\s*\*)\s+(vfisv_\w+)\s*\(", src):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_0901_2702_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_the_boundary():
    names = _declared()
    for n in ("vfisv_create", "vfisv_destroy", "vfisv_synth", "vfisv_invert", "vfisv_check",
              "vfisv_strerror", "vfisv_config_default"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in _declared() if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    import paper_0901_2702_gb300 as v
    monkeypatch.setattr(v, "_LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(v, "_lib", None)
    with pytest.raises(RuntimeError, match="not built"):
        v.load()


def test_host_only_calls(lib):
    """Calls that need no device: error strings and the default config."""
    import paper_0901_2702_gb300 as v
    c = v.vfisv_config_default()
    assert c.max_iter == 50 and c.free_mask == 0x1FF and c.eps0 == 1.0
    assert v.vfisv_strerror(-3).startswith("number of filters")
