"""The C-ABI library builds, loads and exports every symbol include/*.h declares.

CPU only: no compute call is made (rsv_create without a GPU must fail cleanly).
"""
import ctypes
import glob
import os
import re

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _declared():
    names = set()
    for hdr in glob.glob(os.path.join(ROOT, "include", "*.h")):
        text = open(hdr).read()
        text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
        for m in re.finditer(r"\b(rsv_[a-z0-9_]+)\s*\(", text):
            names.add(m.group(1))
    return names


@pytest.fixture(scope="module")
def lib():
    from paper_1603_08114_gb300 import build
    path = build.build()
    return ctypes.CDLL(path)


def test_header_declares_entry_points():
    names = _declared()
    for n in ("rsv_create", "rsv_destroy", "rsv_action", "rsv_force", "rsv_hmc_trajectory",
              "rsv_hmc_chain", "rsv_sync_status", "rsv_last_error"):
        assert n in names


def test_library_exports_every_declared_symbol(lib):
    missing = [n for n in sorted(_declared()) if not hasattr(lib, n)]
    assert not missing, missing


def test_abi_version(lib):
    lib.rsv_abi_version.restype = ctypes.c_int
    text = open(os.path.join(ROOT, "include", "rsv.h")).read()
    v = int(re.search(r"#define RSV_ABI_VERSION (\d+)", text).group(1))
    assert lib.rsv_abi_version() == v


def test_null_context_is_rejected_without_gpu(lib):
    lib.rsv_set_schedule.restype = ctypes.c_int
    lib.rsv_set_schedule.argtypes = [ctypes.c_void_p, ctypes.c_int, ctypes.c_int, ctypes.c_int64]
    assert lib.rsv_set_schedule(None, 0, 0, 0) == 1  # RSV_EINVAL
    lib.rsv_last_error.restype = ctypes.c_char_p
    assert b"context" in lib.rsv_last_error()


def test_create_without_device_fails_cleanly(lib):
    import torch
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    lib.rsv_create.restype = ctypes.c_int
    lib.rsv_create.argtypes = [ctypes.POINTER(ctypes.c_void_p), ctypes.c_int]
    h = ctypes.c_void_p()
    st = lib.rsv_create(ctypes.byref(h), 0)
    assert st in (1, 3)  # RSV_EINVAL (no device) or RSV_ECUDA
    assert not h.value


def test_binding_raises_without_library(monkeypatch, tmp_path):
    from paper_1603_08114_gb300 import rsv
    monkeypatch.setattr(rsv, "_lib", None)
    monkeypatch.setattr(rsv, "lib_path", lambda: str(tmp_path / "missing.so"))
    with pytest.raises(RuntimeError, match="not built"):
        rsv.lib()
