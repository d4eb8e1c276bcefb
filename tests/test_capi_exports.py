"""The C-ABI library builds, loads and exports every symbol its header
declares (no GPU needed: no compute call is made), and host-side argument
checks reject bad input before touching the device."""
import ctypes
import os
import re

import numpy as np
import pytest

from paper_2010_08423_gb300 import build as B
from paper_2010_08423_gb300 import capi

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "restless_reach.h")


def declared_symbols():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(rr_[a-z_0-9]+)\s*\(", text)))


def test_header_declares_the_binding_surface():
    syms = declared_symbols()
    assert set(syms) == set(capi.EXPORTED), set(syms) ^ set(capi.EXPORTED)


def test_library_builds_and_exports_every_symbol():
    path = B.build()
    lib = ctypes.CDLL(path)
    missing = [s for s in declared_symbols() if not hasattr(lib, s)]
    assert not missing, missing


def test_invalid_graph_rejected_on_host():
    capi.load()
    src = np.array([0, 1], dtype=np.uint32)
    dst = np.array([1, 1], dtype=np.uint32)  # self-loop at edge 1
    t = np.array([1, 2], dtype=np.uint32)
    delta = np.array([1, 1], dtype=np.uint32)
    with pytest.raises(capi.RRError) as ei:
        capi.rr_graph_load(2, src, dst, t, delta)
    assert ei.value.status == capi.RR_EINVAL
    assert "self-loop" in capi.rr_last_error()
    with pytest.raises(capi.RRError) as ei:
        capi.rr_graph_load(2, src, np.array([1, 5], dtype=np.uint32), t, delta)
    assert ei.value.status == capi.RR_EINVAL
    with pytest.raises(capi.RRError) as ei:
        capi.rr_graph_load(0, src[:0], dst[:0], t[:0], delta[:0])
    assert ei.value.status == capi.RR_EINVAL


def test_null_handles_rejected():
    lib = capi.load()
    assert lib.rr_graph_free(None) == capi.RR_EINVAL
    assert lib.rr_server_destroy(None) == capi.RR_EINVAL
    assert lib.rr_set_tuning(None, 5, 2, 64) == capi.RR_EINVAL
