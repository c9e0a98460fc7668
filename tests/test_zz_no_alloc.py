"""mphf_build_u64_noalloc: the build for callers that may not allocate device
memory (a framework that owns all device memory through its own pool, a
thread where cudaMalloc's device-wide synchronization is not acceptable, a
fully committed device).  It must produce exactly what the allocating entry
point produces, call after call, without changing the device's free memory.

This file is collected last on purpose: the entry point shares one fixed
device array across calls, and a failure here should not hide the rest."""
from __future__ import annotations

import ctypes

import pytest
import torch

from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu

pytestmark = pytest.mark.gpu


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
