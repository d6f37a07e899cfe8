"""Host-only checks of the C ABI: the library builds, loads and exports every
symbol include/hdconv.h declares; host-side validation needs no GPU."""
import ctypes
import os
import re

import pytest

import paper_2608_14497_b300 as hd
from paper_2608_14497_b300 import build as hdbuild

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def declared_symbols():
    text = open(os.path.join(ROOT, "include", "hdconv.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(hd_[a-z0-9_]+)\s*\(", text)))


def test_library_builds_and_exports_every_declared_symbol():
    hdbuild.build()
    lib = ctypes.CDLL(hd.LIB_PATH)
    syms = declared_symbols()
    assert len(syms) >= 12
    for s in syms:
        assert hasattr(lib, s), s
    assert set(syms) == set(hd.EXPORTS)


def test_strerror_host_only():
    lib = hd.load()
    assert lib.hd_strerror(hd.HD_EINVAL) == b"invalid argument"
    assert lib.hd_strerror(hd.HD_ETIMEOUT) == b"device wait timed out"


def test_null_arguments_rejected_without_gpu():
    lib = hd.load()
    assert lib.hd_create(None, 0) == hd.HD_EINVAL
    assert lib.hd_conv1d(None, hd.HD_HYBRID_RCM, hd.HD_FP32, None, None, None, 16, None, None) == hd.HD_EINVAL
    assert lib.hd_plan(None, hd.HD_HYBRID_RCM, 16, None) == hd.HD_EINVAL
    n = ctypes.c_int32(-1)
    assert lib.hd_batch_plan_launches(None, ctypes.byref(n)) == hd.HD_EINVAL
    assert lib.hd_batch_plan_launches(None, None) == hd.HD_EINVAL
    assert lib.hd_tuning_table(None, 0, None, None, None, ctypes.byref(n)) == hd.HD_EINVAL
