"""mphf_build_u64_noalloc: the build for callers that may not allocate device
memory (a framework that owns all device memory through its own pool, a
thread where cudaMalloc's device-wide synchronization is not acceptable, a
fully committed device).  It must produce exactly what the allocating entry
point produces, call after call, without changing the device's free memory.

This file is collected last on purpose: the entry point shares one fixed
device array across calls, and a failure here should not hide the rest."""
from __future__ import annotations

import ctypes
import os
import subprocess
import sys

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, u32

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _check_against_oracle(N, blob: bytes, keys: torch.Tensor):
    """The serialized result, loaded by the oracle and by the library, gives
    the same values on every key, and they form a bijection onto [0, n)."""
    ref = O.OracleMPHF.deserialize(blob)
    want = ref.query_u64(W.as_uint64_numpy(keys))
    got = u32(N.mphf_query_u64(N.mphf_deserialize(blob), keys))
    assert np.array_equal(got, want)
    assert np.array_equal(np.sort(want), np.arange(keys.numel(), dtype=np.uint32))


def test_noalloc_build_matches_mphf_build_on_consecutive_calls():
    N = need_gpu()
    cases = [(50_000, 1, {}), (777, 2, {"lam": 3.0, "gamma": 1, "remap": 1})]
    free_before_second = None
    for i, (n, seed, params) in enumerate(cases):
        keys = W.u64_keys(n, seed).cuda()
        want = N.mphf_serialize(N.mphf_build(keys, N.mphf_default_params(**params)))
        torch.cuda.synchronize()
        if i == 1:
            free_before_second = torch.cuda.mem_get_info()[0]
        got = N.mphf_build_u64_noalloc(keys, N.mphf_default_params(**params))
        torch.cuda.synchronize()
        if i == 1:
            assert torch.cuda.mem_get_info()[0] == free_before_second   # no device allocation
        assert got == want, f"call {i}: structures differ"


@pytest.mark.parametrize("n,params", [
    (65_536, {}),                                                        # the largest n, default layout
    (65_536, {"slots_override": 1024, "alpha": 0.8, "remap": 1}),        # 80 parts, one CTA per part
    (1, {}),                                                             # the smallest n
])
def test_noalloc_build_at_its_limits_matches_mphf_build_and_the_oracle(n, params):
    N = need_gpu()
    keys = W.u64_keys(n, 40 + n % 7).cuda()
    p = N.mphf_default_params(**params)
    want = N.mphf_serialize(N.mphf_build(keys, p))
    got = N.mphf_build_u64_noalloc(keys, p)
    assert got == want
    if params.get("slots_override"):
        assert N.mphf_info(N.mphf_deserialize(got))["P"] > 64
    _check_against_oracle(N, got, keys)


def test_noalloc_build_rejects_too_many_keys():
    N = need_gpu()
    lib = N.load()
    keys = W.u64_keys(65_537, 3).cuda()
    p = N.mphf_default_params()
    need = ctypes.c_size_t()
    buf = ctypes.create_string_buffer(1 << 20)
    rc = lib.mphf_build_u64_noalloc(ctypes.byref(p), keys.data_ptr(), keys.numel(), buf, 1 << 20,
                                    ctypes.byref(need), torch.cuda.current_stream().cuda_stream)
    assert rc == N.MPHF_ERR_CAPACITY
    assert b"65536" in lib.mphf_last_error()


def test_noalloc_build_rejects_a_layout_larger_than_its_array():
    """65,536 keys in one part of 2^20 slots: the per-part slot owners and
    hashes alone need 12 MiB, more than the fixed 8 MiB array."""
    N = need_gpu()
    lib = N.load()
    keys = W.u64_keys(65_536, 4).cuda()
    p = N.mphf_default_params(slots_override=1 << 20)
    need = ctypes.c_size_t()
    buf = ctypes.create_string_buffer(1 << 22)
    rc = lib.mphf_build_u64_noalloc(ctypes.byref(p), keys.data_ptr(), keys.numel(), buf, 1 << 22,
                                    ctypes.byref(need), torch.cuda.current_stream().cuda_stream)
    assert rc == N.MPHF_ERR_CAPACITY
    assert b"scratch array" in lib.mphf_last_error()


_FRESH = r"""
import sys, torch
sys.path.insert(0, sys.argv[1])
from paper_2502_15539_gb300 import native as N, workloads as W
N.load()
keys = W.u64_keys(30000, 9).cuda()
torch.cuda.synchronize()
f0 = torch.cuda.mem_get_info()[0]
a = N.mphf_build_u64_noalloc(keys)          # the first call into the builder in this process
torch.cuda.synchronize()
f1 = torch.cuda.mem_get_info()[0]
b = N.mphf_build_u64_noalloc(keys)
torch.cuda.synchronize()
f2 = torch.cuda.mem_get_info()[0]
c = N.mphf_serialize(N.mphf_build(keys))
print("first-call-drop", f0 - f1, "second-call-drop", f1 - f2)
assert a == b == c, "structures differ"
assert f2 == f1, "the second call changed the free device memory"
print("ok")
"""


def test_noalloc_build_as_the_first_builder_call_of_a_fresh_process():
    """In a new process whose first builder call is this entry point, the
    module (and with it the fixed array) is loaded by that call; the second
    call then allocates nothing, and both equal mphf_build's structure."""
    need_gpu()
    res = subprocess.run([sys.executable, "-c", _FRESH, ROOT], capture_output=True, text=True, timeout=300)
    assert res.returncode == 0, res.stdout + res.stderr
    assert res.stdout.strip().endswith("ok")
