"""Host-side checks of the C ABI: the library loads, exports every declared
entry point, and its host logic (parameter rule, argument and format
validation) behaves; no GPU is needed."""
from __future__ import annotations

import ctypes
import os
import re

import pytest

from oracle import oracle as O
from paper_2502_15539_gb300 import build_ext
from paper_2502_15539_gb300 import native as N

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module")
def lib():
    build_ext.build()
    return N.load()


def declared_functions():
    text = open(os.path.join(ROOT, "include", "mphf.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(mphf_\w+)\s*\(", text)))


def test_every_declared_symbol_is_exported(lib):
    names = declared_functions()
    assert "mphf_build" in names and "mphf_query_u64" in names and "mphf_free" in names
    for name in names:
        assert hasattr(lib, name), name
    assert set(names) == set(N.SIGNATURES), "binding and header disagree"


def test_default_params(lib):
    p = N.mphf_default_params()
    assert p.lambda_ == 3.5 and p.alpha == 0.99
    assert p.gamma == N.MPHF_GAMMA_CUBIC and p.remap == N.MPHF_REMAP_CLEF
    assert p.C & 1 and p.evict_mult == 10


@pytest.mark.parametrize("n", [1, 7, 23, 1000, 80_000, 100_000, 300_000, 10**6, 10**7, 3 * 10**8, 10**9,
                               4_000_000_000])
@pytest.mark.parametrize("lam", [3.0, 3.5, 4.0])
def test_layout_rule_matches_the_oracle(lib, n, lam):
    """Both implementations of the parameter rule (Sec. 3.1) pick the same layout."""
    info = N.mphf_layout(n, N.mphf_default_params(lam=lam))
    L = O.layout_for(n, lam, 0.99)
    assert (info["P"], info["S"], info["B"], info["reduce"]) == (L.P, L.S, L.B, L.reduce)
    assert info["remap_len"] == L.P * L.S - n


def test_layout_at_1e9(lib):
    info = N.mphf_layout(10**9)
    assert (info["P"], info["S"], info["B"]) == (964, 1 << 20, 296_598)
    assert abs(info["bits_per_key"] - 2.41) < 0.01


def test_argument_errors_need_no_gpu(lib):
    assert lib.mphf_query_u64(None, None, 5, None, None) == N.MPHF_ERR_ARG
    out = ctypes.c_void_p()
    assert lib.mphf_deserialize(b"not a structure" * 10, 150, ctypes.byref(out)) == N.MPHF_ERR_FORMAT
    assert out.value is None
    assert lib.mphf_deserialize(None, 0, ctypes.byref(out)) == N.MPHF_ERR_ARG
    p = N.mphf_default_params()
    assert lib.mphf_build(ctypes.byref(p), 0, None, None, 10, None, ctypes.byref(out)) == N.MPHF_ERR_ARG
    info = N.mphf_info_t()
    assert lib.mphf_layout(ctypes.byref(p), 0, ctypes.byref(info)) == N.MPHF_ERR_ARG
    lib.mphf_free(None)
    assert lib.mphf_lookup_u64(None, None, 5, None, 4, None, None) == N.MPHF_ERR_ARG
    assert lib.mphf_set_l2_fetch_granularity(129, None) == N.MPHF_ERR_ARG
    assert lib.mphf_set_l2_fetch_granularity(-1, None) == N.MPHF_ERR_ARG
    assert lib.mphf_strerror(N.MPHF_ERR_DUP_KEYS) == b"duplicate keys"
    assert b"NULL" in lib.mphf_last_error() or lib.mphf_last_error()


def test_header_validation_rejects_corruption(lib):
    """The library's format reader rejects what the oracle's writer never writes."""
    import numpy as np
    from paper_2502_15539_gb300 import workloads as W
    ref = O.OracleMPHF.build_u64(W.as_uint64_numpy(W.u64_keys(3000)))
    blob = bytearray(ref.serialize())
    out = ctypes.c_void_p()
    for off, val in [(8, 2), (16, 2), (20, 7), (24, 5)]:   # version, gamma, remap, reduce
        bad = bytearray(blob)
        bad[off:off + 4] = int(val).to_bytes(4, "little")
        assert lib.mphf_deserialize(bytes(bad), len(bad), ctypes.byref(out)) == N.MPHF_ERR_FORMAT
    bad = bytearray(blob)
    bad[64:72] = (2).to_bytes(8, "little")                  # even mixing constant
    assert lib.mphf_deserialize(bytes(bad), len(bad), ctypes.byref(out)) == N.MPHF_ERR_FORMAT
    assert lib.mphf_deserialize(bytes(blob[:-1]), len(blob) - 1, ctypes.byref(out)) == N.MPHF_ERR_FORMAT


def test_device_view_argument_errors(lib):
    v = N.mphf_view_t()
    assert lib.mphf_device_view(None, ctypes.byref(v)) == N.MPHF_ERR_ARG


def test_device_header_compiles_in_a_caller():
    """include/mphf_device.cuh is self-contained: a caller's translation unit
    that includes it cross-compiles for sm_103a."""
    from tests.device_api_common import compile_caller, nvcc
    import tempfile
    if nvcc() is None:
        pytest.skip("nvcc not found")
    with tempfile.TemporaryDirectory() as d:
        compile_caller(os.path.join(d, "caller.o"), shared=False)
