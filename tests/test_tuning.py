"""Host logic of the autotuner (no GPU): the cache key, the JSON-lines cache,
and the argument checks of tho_plan_tuned that run before any CUDA call."""
import ctypes
import json

import pytest
import torch

from paper_2602_14449_gb300 import build as tho_build
from paper_2602_14449_gb300 import tho

F, C = tho.THO_F64, tho.THO_C128


@pytest.fixture(scope="module")
def lib():
    tho_build.build()
    return tho.load()


def test_key_names_device_mode_and_shape_buckets(lib):
    k = tho.tune_key([(1 << 22, 128, 32)], torch.complex128, tho.THO_PREC_FP64_EMU, 0, "NVIDIA GB300")
    assert k == "NVIDIA GB300|c128|emu|f0|q88:128:32"  # floor(4 log2 2^22) = 88
    assert tho.tune_key([(4096, 16, 4)], torch.float64, tho.THO_PREC_FP64, tho.THO_FLAG_P_MLU, "d") == \
        "d|f64|fp64|f4|q48:16:4"


@pytest.mark.parametrize("n", [1, 2, 3, 5, 1000, 4095, 4096, 4097, 6000, 1 << 20, (1 << 22) + 12345, (1 << 40) + 7])
def test_n_bucket_is_floor_of_four_log2(lib, n):
    import math
    want = math.floor(4 * math.log2(n))
    # Away from the irrational quarter-octave boundaries the float log is exact enough.
    got = int(tho.tune_key([(n, 0, 1)], torch.float64, 0, 1, "d").split("|")[-1].split(":")[0][1:])
    assert got == want


def test_key_buckets_nearby_sizes_and_hashes_large_batches(lib):
    key = lambda shapes: tho.tune_key(shapes, torch.float64, 0, 0, "dev")
    assert key([(1 << 20, 64, 16)]) == key([((1 << 20) + 1000, 64, 16)])
    assert key([(1 << 20, 64, 16)]) != key([(1 << 21, 64, 16)])
    assert key([(1 << 20, 64, 16)]) != key([(1 << 20, 32, 16)])
    small = key([(20000, 8, 4), (30000, 16, 8)])
    assert small.endswith("q57:8:4,q59:16:8")
    big = [(16384 + 997 * i, 8 * (1 + i % 4), 4 * (1 + i % 3)) for i in range(40)]
    kb = key(big)
    assert kb.split("|")[-1].startswith("batch40:") and len(kb.split(":")[-1]) == 16
    assert kb == key(list(big))
    assert kb != key(big[::-1])  # the batch key follows the problem order


def test_key_sanitizes_the_device_name_and_checks_arguments(lib):
    assert tho.tune_key([(100, 4, 4)], torch.float64, 0, 0, 'a"b\\c|d').startswith("a_b_c_d|")
    arr = (tho.Desc * 1)(tho.Desc(100, 4, 4, F, 0, 0))
    small = ctypes.create_string_buffer(8)
    assert lib.tho_tune_key(arr, 1, b"dev", small, len(small)) == tho.THO_ERR_ARG
    assert lib.tho_tune_key(None, 1, b"dev", small, len(small)) == tho.THO_ERR_ARG
    assert lib.tho_tune_key(arr, 0, b"dev", small, len(small)) == tho.THO_ERR_ARG


def test_cache_round_trip_last_entry_wins(lib, tmp_path):
    path = str(tmp_path / "tune.jsonl")
    assert tho.tune_cache_get(path, "k1") is None  # missing file: no entries
    tho.tune_cache_put(path, "k1", (128, 303, 0), 101.25)
    tho.tune_cache_put(path, "k2", (64, 152, 1), 7.5)
    assert tho.tune_cache_get(path, "k1") == ((128, 303, 0), 101.25)
    tho.tune_cache_put(path, "k1", (256, 607, 1), 99.0)
    assert tho.tune_cache_get(path, "k1") == ((256, 607, 1), 99.0)
    assert tho.tune_cache_get(path, "k2") == ((64, 152, 1), 7.5)
    assert tho.tune_cache_get(path, "k3") is None
    rows = [json.loads(line) for line in open(path)]  # every line is a JSON object
    assert [r["key"] for r in rows] == ["k1", "k2", "k1"]
    assert rows[-1] == {"key": "k1", "leaf_rows": 256, "split_chunks": 607, "balance": 1, "ms": 99.0}


def test_cache_skips_lines_that_do_not_parse(lib, tmp_path):
    path = tmp_path / "tune.jsonl"
    path.write_text('garbage\n{"key": "k1", "leaf_rows": 128}\n'
                    '{"key": "k1", "leaf_rows": 1.5, "split_chunks": 3, "balance": 0, "ms": 1}\n'
                    '{"key": "k1", "leaf_rows": 64, "split_chunks": -3, "balance": 0, "ms": 1}\n'
                    '{"key": "k1", "leaf_rows": 64, "split_chunks": 3, "balance": 2, "ms": 1}\n'
                    '{"key": "k1", "leaf_rows": 64, "split_chunks": 300, "balance": 1, "ms": 2.5}\n'
                    '{"key": "k1", "leaf_rows": 128, "split_chunks": 30')  # truncated last line
    assert tho.tune_cache_get(str(path), "k1") == ((64, 300, 1), 2.5)


def test_cache_put_rejects_keys_that_would_break_the_line(lib, tmp_path):
    path = str(tmp_path / "tune.jsonl")
    t = tho.Tuning(128, 10, 0)
    for bad in (b'a"b', b"a\\b", b"a\nb"):
        assert lib.tho_tune_cache_put(path.encode(), bad, ctypes.byref(t), 1.0) == tho.THO_ERR_ARG
    assert lib.tho_tune_cache_put(None, b"k", ctypes.byref(t), 1.0) == tho.THO_ERR_ARG
    assert lib.tho_tune_cache_put(str(tmp_path / "no" / "dir.jsonl").encode(), b"k", ctypes.byref(t),
                                  1.0) == tho.THO_ERR_ARG
    found = ctypes.c_int32(7)
    assert lib.tho_tune_cache_get(None, b"k", ctypes.byref(t), None, ctypes.byref(found)) == tho.THO_ERR_ARG


def _plan_tuned(lib, desc, leaf, split, balance=0):
    arr = (tho.Desc * 1)(tho.Desc(*desc))
    t = tho.Tuning(leaf, split, balance)
    h = ctypes.c_void_p()
    return lib.tho_plan_tuned(arr, 1, ctypes.byref(t), ctypes.byref(h))


def test_plan_tuned_rejects_bad_choices_on_the_host(lib):
    d = (1 << 16, 16, 8, F, 0, 0)
    for leaf in (1, 32, 100, 512, -64):
        assert _plan_tuned(lib, d, leaf, 0) == tho.THO_ERR_ARG
    for split in (-1, tho.THO_TUNE_MAX_SPLIT + 1):
        assert _plan_tuned(lib, d, 0, split) == tho.THO_ERR_ARG
    for balance in (-1, 2):
        assert _plan_tuned(lib, d, 0, 0, balance) == tho.THO_ERR_ARG
    # A complex FP64 leaf panel of 256 rows with k0 = 128 staged beside k = 32
    # columns needs more shared memory than a CTA has.
    assert _plan_tuned(lib, (1 << 16, 128, 32, C, 0, 0), 256, 0) == tho.THO_ERR_UNSUPPORTED
    # Descriptor errors come first, as in tho_plan.
    assert _plan_tuned(lib, (10, 6, 5, F, 0, 0), 128, 0) == tho.THO_ERR_SHAPE
    assert lib.tho_plan_tuning(None, None) == tho.THO_ERR_ARG
