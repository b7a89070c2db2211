"""CPU checks of the C ABI library: it builds, loads without a GPU, and exports
every function include/lodgs.h declares (no compute calls are made)."""
import ctypes as C
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    src = open(os.path.join(ROOT, "include", "lodgs.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(lodgs_[a-z0-9_]+)\s*\(", src)))


def test_library_builds_and_exports_every_declared_symbol():
    from paper_2507_01110_b300 import build
    path = build.build()
    lib = C.CDLL(path)
    names = _declared()
    assert len(names) >= 12
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_declares_the_same_symbols():
    from paper_2507_01110_b300 import _lib
    assert sorted(_lib.EXPORTED) == _declared()


def test_binding_fails_loudly_without_library(tmp_path, monkeypatch):
    from paper_2507_01110_b300 import _lib
    monkeypatch.setattr(_lib, "LIB_PATH", str(tmp_path / "missing.so"))
    monkeypatch.setattr(_lib, "_lib", None)
    try:
        _lib.lib()
    except _lib.LodgsError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("loading a missing library must raise")


def test_version_and_errors_without_gpu():
    from paper_2507_01110_b300 import _lib
    L = _lib.lib()
    assert b"lodgs" in L.lodgs_version()
    # argument validation happens before any CUDA call
    h = C.c_void_p()
    p = _lib.BuildParams(0.0, 1.0)
    rc = L.lodgs_build_hierarchy(None, 0, 0, 0, C.byref(p), C.byref(h))
    assert rc == _lib.LODGS_E_INVALID and h.value is None
    assert b"build_hierarchy" in L.lodgs_last_error()


def test_fault_injection_hook_validates_its_site():
    from paper_2507_01110_b300 import _lib
    lib = _lib.lib()
    assert lib.lodgs_debug_inject_fault(0, 0) == _lib.LODGS_E_INVALID
    assert lib.lodgs_debug_inject_fault(_lib.FAULT_ALLOC, -1) == _lib.LODGS_OK
    assert lib.lodgs_debug_inject_fault(_lib.FAULT_STREAM, -1) == _lib.LODGS_OK


def test_binding_constants_match_the_header():
    """Every #define of include/lodgs.h that the binding mirrors has the
    header's value (status codes, batch bound, fault sites, densify ops)."""
    from paper_2507_01110_b300 import _lib
    src = open(os.path.join(ROOT, "include", "lodgs.h")).read()
    defs = {m.group(1): int(m.group(2).replace(" ", ""))
            for m in re.finditer(r"#define\s+(LODGS_[A-Z0-9_]+)\s+\(?\s*(-?\s*\d+)\s*\)?\s*(?:/\*|$)", src, flags=re.M)}
    mirrored = {"LODGS_OK", "LODGS_E_INVALID", "LODGS_E_OOM", "LODGS_E_CUDA", "LODGS_E_TIMEOUT", "LODGS_E_STATE",
                "LODGS_E_CAPACITY", "LODGS_SELECT_BATCH_MAX"}
    assert mirrored <= set(defs), mirrored - set(defs)
    for name in mirrored:
        assert getattr(_lib, name) == defs[name], name
    for name in ("FAULT_STREAM", "FAULT_ALLOC", "FAULT_RENDER"):
        assert getattr(_lib, name) == defs["LODGS_" + name], name
