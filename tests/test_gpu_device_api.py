"""The device API (include/mphf_device.cuh): a caller's own kernels, compiled
apart from libmphf, evaluate structures through mphf_device_view() and must
give the oracle's values bit for bit (Sec. 3.1 Eq. slot, Sec. 3.3 gamma,
Sec. 3.4 remap), for every layout the library builds."""
from __future__ import annotations

import ctypes

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.device_api_common import caller_library
from tests.gpu_common import need_gpu, oracle_structure, u32

pytestmark = pytest.mark.gpu

CASES = [
    (1, {}),
    (1000, {}),
    (4097, {"gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),
    (30_000, {"slots_override": 2048, "alpha": 0.9}),                       # POW2, 17 parts
    (30_000, {"slots_override": 3001, "alpha": 0.9}),                       # x mod S
    (200_000, {}),                                                          # MOD layout
    (10**6, {}),                                                            # P=4, S=2^18
    (10**6, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),   # Fast
]


def ids(c):
    n, p = c
    return f"n{n}-" + "-".join(f"{k}{v}" for k, v in sorted(p.items()))


def caller():
    lib = ctypes.CDLL(caller_library())
    vp = ctypes.c_void_p
    for name in ("caller_eval_u64", "caller_count_u64", "caller_slot_u64", "caller_eval_u64_wide",
                 "caller_eval_u64_n4"):
        getattr(lib, name).argtypes = [vp, vp, ctypes.c_uint64, vp, vp]
        getattr(lib, name).restype = ctypes.c_int
    lib.caller_eval_bytes.argtypes = [vp, vp, vp, ctypes.c_uint64, vp, vp]
    lib.caller_eval_bytes.restype = ctypes.c_int
    return lib


def stream():
    return ctypes.c_void_p(torch.cuda.current_stream().cuda_stream)


@pytest.mark.parametrize("case", CASES, ids=[ids(c) for c in CASES])
def test_caller_kernel_matches_oracle(case):
    N = need_gpu()
    lib = caller()
    n, params = case
    ref, blob = oracle_structure(n, 0, **params)
    m = N.mphf_deserialize(blob)
    view = N.mphf_device_view(m)
    assert view.n == n and view.P == ref.layout.P and view.S == ref.layout.S and view.key_kind == 0
    keys = W.u64_keys(n, 0)
    q = torch.cat([keys[W.permutation(n, 1)], W.nonmember_u64_keys(max(n // 4, 17), n, 0)]).cuda()
    out = torch.empty(q.numel(), dtype=torch.int32, device="cuda")
    assert lib.caller_eval_u64(ctypes.byref(view), q.data_ptr(), q.numel(), out.data_ptr(), stream()) == 0
    want = ref.query_u64(W.as_uint64_numpy(q.cpu()))
    got = u32(out)
    assert np.array_equal(got, want), f"{int((got != want).sum())} mismatches"
    assert np.array_equal(got, u32(N.mphf_query_u64(m, q)))

    wide = torch.empty(q.numel(), dtype=torch.int64, device="cuda")
    assert lib.caller_eval_u64_wide(ctypes.byref(view), q.data_ptr(), q.numel(), wide.data_ptr(), stream()) == 0
    assert np.array_equal(wide.cpu().numpy().view(np.uint64), want)

    grouped = torch.empty(q.numel(), dtype=torch.int32, device="cuda")   # 4 keys per thread, ragged tail
    assert lib.caller_eval_u64_n4(ctypes.byref(view), q.data_ptr(), q.numel(), grouped.data_ptr(), stream()) == 0
    assert np.array_equal(u32(grouped), want)

    slots = torch.empty(q.numel(), dtype=torch.int64, device="cuda")
    assert lib.caller_slot_u64(ctypes.byref(view), q.data_ptr(), q.numel(), slots.data_ptr(), stream()) == 0
    assert np.array_equal(slots.cpu().numpy().view(np.uint64), ref.slots_u64(W.as_uint64_numpy(q.cpu())))


@pytest.mark.parametrize("n", [1000, 10**6])
def test_fused_consumer_counts_each_value_once(n):
    """The lookup fused into a consumer kernel: each member key increments the
    counter its value names; a perfect hash leaves every counter at one."""
    N = need_gpu()
    lib = caller()
    _, blob = oracle_structure(n, 0)
    m = N.mphf_deserialize(blob)
    view = N.mphf_device_view(m)
    keys = W.u64_keys(n, 0).cuda()
    counts = torch.zeros(n, dtype=torch.int32, device="cuda")
    assert lib.caller_count_u64(ctypes.byref(view), keys.data_ptr(), n, counts.data_ptr(), stream()) == 0
    assert bool((counts == 1).all())


@pytest.mark.parametrize("n,params", [(37, {}), (100_000, {}),
                                      (50_000, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),
                                      (20_000, {"hash128": 1})])
def test_caller_string_kernel_matches_oracle(n, params):
    N = need_gpu()
    lib = caller()
    ids_ = torch.arange(n)
    data, off = W.strings(ids_, seed=3)
    ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=8, **params)
    m = N.mphf_deserialize(ref.serialize())
    view = N.mphf_device_view(m)
    assert view.key_kind == 1 and view.hash128 == params.get("hash128", 0)
    qd, qo = W.strings(torch.cat([ids_[W.permutation(n, 1)], torch.arange(n, n + n // 4 + 5)]), seed=3)
    dd, do = qd.cuda(), qo.cuda()
    out = torch.empty(qo.numel() - 1, dtype=torch.int32, device="cuda")
    assert lib.caller_eval_bytes(ctypes.byref(view), dd.data_ptr(), do.data_ptr(), out.numel(),
                                 out.data_ptr(), stream()) == 0
    got = u32(out)
    assert np.array_equal(got, ref.query_bytes(qd.numpy(), qo.numpy().astype(np.uint64)))


@pytest.mark.parametrize("case", CASES, ids=[ids(c) for c in CASES])
def test_fused_lookup_reads_the_table_at_the_oracle_value(case):
    """mphf_lookup_u64: out[i] = table[h(q[i])], h the oracle's value of each key."""
    N = need_gpu()
    n, params = case
    ref, blob = oracle_structure(n, 0, **params)
    m = N.mphf_deserialize(blob)
    keys = W.u64_keys(n, 0)
    q = torch.cat([keys[W.permutation(n, 1)], W.nonmember_u64_keys(max(n // 4, 17), n, 0)])
    want = ref.query_u64(W.as_uint64_numpy(q)).astype(np.int64)
    gen = torch.Generator().manual_seed(n)
    for dtype in (torch.int32, torch.int64):
        table = torch.randint(-2**31, 2**31 - 1, (n,), generator=gen, dtype=torch.int64).to(dtype)
        got = N.mphf_lookup_u64(m, q.cuda(), table.cuda()).cpu()
        assert torch.equal(got, table[torch.from_numpy(want)])


@pytest.mark.parametrize("count", [0, 1, 2047, 2048, 2049, 6143, 10_001])
def test_fused_lookup_ragged_counts(count):
    N = need_gpu()
    n = 5000
    ref, blob = oracle_structure(n, 0)
    m = N.mphf_deserialize(blob)
    q = W.u64_keys(count, 9)   # mostly non-members: every key still reads some element
    table = torch.arange(n, dtype=torch.int64) * 3 + 1
    out = torch.full((count,), -7, dtype=torch.int64, device="cuda")
    N.mphf_lookup_u64(m, q.cuda(), table.cuda(), out)
    want = table[torch.from_numpy(ref.query_u64(W.as_uint64_numpy(q)).astype(np.int64))]
    assert torch.equal(out.cpu(), want)


def test_fused_lookup_argument_errors():
    N = need_gpu()
    _, blob = oracle_structure(1000, 0)
    m = N.mphf_deserialize(blob)
    lib = N.load()
    q = W.u64_keys(100, 0).cuda()
    table = torch.zeros(1000, dtype=torch.int32, device="cuda")
    out = torch.zeros(100, dtype=torch.int32, device="cuda")
    assert lib.mphf_lookup_u64(m.handle, q.data_ptr(), 100, table.data_ptr(), 2, out.data_ptr(), None) == N.MPHF_ERR_ARG
    assert lib.mphf_lookup_u64(m.handle, q.data_ptr() + 4, 10, table.data_ptr(), 4, out.data_ptr(), None) == N.MPHF_ERR_ARG
    assert lib.mphf_lookup_u64(m.handle, q.data_ptr(), 10, table.data_ptr() + 2, 4, out.data_ptr(), None) == N.MPHF_ERR_ARG
    data, off = W.strings(torch.arange(50), seed=1)
    sref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=2)
    sm = N.mphf_deserialize(sref.serialize())
    assert lib.mphf_lookup_u64(sm.handle, q.data_ptr(), 10, table.data_ptr(), 4, out.data_ptr(), None) == N.MPHF_ERR_ARG
