"""The C ABI library loads, exports every symbol include/tho.h declares, and
rejects bad arguments on the host (no GPU needed for any of this)."""
import ctypes
import os
import re
import subprocess

import pytest

from paper_2602_14449_gb300 import build as tho_build
from paper_2602_14449_gb300 import tho

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tho.h")


@pytest.fixture(scope="module")
def lib():
    tho_build.build()
    return tho.load()


def _declared():
    src = open(HEADER).read()
    src = re.sub(r"/\*.*?\*/", "", src, flags=re.S)
    return sorted(set(re.findall(r"\b(tho_[a-z_]+)\s*\(", src)))


def test_header_declares_the_binding_surface():
    assert set(_declared()) == set(tho.EXPORTED)


def test_every_declared_symbol_is_exported(lib):
    out = subprocess.run(["nm", "-D", "--defined-only", tho.LIB_PATH], capture_output=True, text=True,
                         check=True).stdout
    exported = set(re.findall(r"\bT (tho_[a-z_]+)\b", out))
    for name in _declared():
        assert name in exported, name
        assert hasattr(lib, name)


def _plan(lib, descs):
    arr = (tho.Desc * max(len(descs), 1))(*[tho.Desc(*d) for d in descs])
    h = ctypes.c_void_p()
    return lib.tho_plan(arr, len(descs), ctypes.byref(h))


def test_shape_and_argument_errors(lib):
    F, C = tho.THO_F64, tho.THO_C128
    assert _plan(lib, [(10, 6, 5, F, 0, 0)]) == tho.THO_ERR_SHAPE        # k0 + k > n
    assert _plan(lib, [(10, 0, 5, F, 0, 0)]) == tho.THO_ERR_SHAPE        # k0 = 0 without the flag
    assert _plan(lib, [(10, 2, 0, F, 0, 0)]) == tho.THO_ERR_SHAPE        # k = 0
    assert _plan(lib, [(100, 4, 33, F, 0, 0)]) == tho.THO_ERR_UNSUPPORTED  # k > THO_MAX_K
    assert _plan(lib, [(1000, 129, 4, F, 0, 0)]) == tho.THO_ERR_UNSUPPORTED  # k0 > THO_MAX_K0
    assert _plan(lib, [(100, 4, 4, 7, 0, 0)]) == tho.THO_ERR_ARG         # unknown dtype
    assert _plan(lib, [(100, 4, 4, F, 5, 0)]) == tho.THO_ERR_ARG         # unknown precision
    assert _plan(lib, [(100, 4, 4, F, 0, 0x80)]) == tho.THO_ERR_ARG      # unknown flag
    both = tho.THO_FLAG_P_MLU | tho.THO_FLAG_P_POLAR
    assert _plan(lib, [(100, 4, 4, F, 0, both)]) == tho.THO_ERR_ARG      # two choices of P at once
    assert _plan(lib, [(100, 4, 4, F, 0, 0), (100, 4, 4, C, 0, 0)]) == tho.THO_ERR_ARG  # mixed dtypes
    assert _plan(lib, []) == tho.THO_ERR_ARG
    h = ctypes.c_void_p()
    assert lib.tho_plan(None, 1, ctypes.byref(h)) == tho.THO_ERR_ARG
    assert lib.tho_orth(None, None, 0, None, 0, None, 0, None, None, None) == tho.THO_ERR_ARG
    assert lib.tho_orth_batched(None, None, 0, None) == tho.THO_ERR_ARG
    assert lib.tho_plan_status(None) == tho.THO_ERR_ARG
    assert lib.tho_plan_expire_wait(None, 10, None) == tho.THO_ERR_ARG
    assert lib.tho_plan_destroy(None) == tho.THO_OK
    assert lib.tho_plan_workspace_bytes(None) == 0


def test_status_strings(lib):
    for code in range(11):
        s = lib.tho_status_string(code).decode()
        assert s and s != "unknown status"
    assert lib.tho_status_string(99).decode() == "unknown status"


def test_product_code_never_touches_the_oracle():
    pkg = os.path.join(ROOT, "paper_2602_14449_gb300")
    for dirpath, _, files in os.walk(pkg):
        if "_build" in dirpath:
            continue
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h", ".cpp")):
                text = open(os.path.join(dirpath, f)).read()
                assert "import oracle" not in text and "from oracle" not in text, f
                assert "liboracle" not in text and "tho_oracle" not in text, f


def test_binding_fails_loudly_without_library(tmp_path):
    tho_mod = tho
    saved = tho_mod._lib
    try:
        tho_mod._lib = None
        with pytest.raises(RuntimeError):
            tho_mod.load(str(tmp_path / "missing.so"))
    finally:
        tho_mod._lib = saved


def test_block_plan_argument_errors(lib):
    """tho_blocks_plan rejects bad block lists before touching the device."""
    h = ctypes.c_void_p()

    def plan(n, kb):
        arr = (ctypes.c_int32 * len(kb))(*kb)
        return lib.tho_blocks_plan(n, arr, len(kb), tho.THO_F64, tho.THO_PREC_FP64, ctypes.byref(h))

    assert lib.tho_blocks_plan(100, None, 1, 0, 0, ctypes.byref(h)) == tho.THO_ERR_ARG
    assert plan(100, []) == tho.THO_ERR_ARG
    assert plan(1000, [8, 33]) == tho.THO_ERR_UNSUPPORTED      # a block wider than THO_MAX_K
    assert plan(1000, [0, 8]) == tho.THO_ERR_UNSUPPORTED
    assert plan(1000, [64, 65, 8]) == tho.THO_ERR_UNSUPPORTED  # the last step's k0 = 129 > THO_MAX_K0
    assert plan(20, [16, 16]) == tho.THO_ERR_SHAPE             # K > n
    assert lib.tho_blocks_destroy(None) == tho.THO_OK
