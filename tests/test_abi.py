"""The C ABI library builds, loads and exports every symbol include/pmplus.h declares (no GPU needed)."""
import ctypes
import os
import re

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    src = open(os.path.join(ROOT, "include", "pmplus.h")).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(pmp_[a-z0-9_]+)\s*\(", src)))


def test_header_declares_the_boundary():
    names = declared_symbols()
    for required in ("pmp_key_create", "pmp_key_destroy", "pmp_key_export", "pmp_hash32",
                     "pmp_hash64", "pmp_hash_batch32", "pmp_hash_batch64"):
        assert required in names


def test_library_exports_every_declared_symbol():
    from paper_1609_09840_gb300 import build

    lib_path = build.build()
    lib = ctypes.CDLL(lib_path)
    for name in declared_symbols():
        assert hasattr(lib, name), name
    # host-only entry points work without a device
    lib.pmp_strerror.restype = ctypes.c_char_p
    assert lib.pmp_strerror(0) == b"ok"
    lib.pmp_hash_scratch_bytes.restype = ctypes.c_size_t
    lib.pmp_hash_scratch_bytes.argtypes = [ctypes.c_int, ctypes.c_uint64]
    assert lib.pmp_hash_scratch_bytes(32, 100) == 0          # one level: no scratch
    assert lib.pmp_hash_scratch_bytes(32, 1 << 30) > 0       # five levels
    assert lib.pmp_hash_scratch_bytes(31, 100) == 0          # bad width


def test_binding_fails_loudly_without_library(monkeypatch, tmp_path):
    from paper_1609_09840_gb300 import native

    monkeypatch.setattr(native, "_lib", None)
    monkeypatch.setattr(native, "LIB_PATH", str(tmp_path / "missing.so"))
    try:
        native.load()
    except RuntimeError as e:
        assert "missing" in str(e)
    else:
        raise AssertionError("load() must raise when the CUDA library is absent")
