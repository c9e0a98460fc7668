"""The windowed query against the oracle, element by element.

mphf_query_u64_windowed cuts the pilot array into W byte ranges and streams
the keys once per range; its values must be the oracle's evaluation of the
same structure (Sec. 3.1 Eq. partbucket and Eq. slot, Sec. 3.4 remap), for
every layout, every W, and chunks that leave ragged tails.  Small windows
and chunks put many passes and chunks on small structures, so the oracle
finishes in seconds."""
from __future__ import annotations

import threading

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, oracle_structure, u32

pytestmark = pytest.mark.gpu

LAYOUTS = [
    (30_000, {"slots_override": 2048, "alpha": 0.9}),                                  # 17 parts, POW2, CLEF
    (30_000, {"slots_override": 3001, "alpha": 0.9}),                                  # x mod S, many parts
    (20_000, {"slots_override": 1024, "alpha": 0.9, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),
    (200_000, {}),                                                                     # one part, x mod S
    (10**6, {}),                                                                       # P = 4, S = 2^18
    (10**6, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),              # Fast
]


def _query_stream(n: int) -> torch.Tensor:
    keys = W.u64_keys(n, 0)
    return torch.cat([keys[W.permutation(n, 1)], W.nonmember_u64_keys(n // 4 + 3, n, 0)])


@pytest.mark.parametrize("n,params", LAYOUTS)
@pytest.mark.parametrize("windows", [2, 3, 7])
def test_windowed_query_matches_oracle(n, params, windows):
    N = need_gpu()
    ref, blob = oracle_structure(n, 0, **params)
    m = N.mphf_deserialize(blob)
    info = N.mphf_info(m)
    nbkt = info["P"] * info["B"]
    window_bytes = -(-nbkt // windows)                   # ceil: exactly `windows` ranges
    q = _query_stream(n)
    want = ref.query_u64(W.as_uint64_numpy(q))
    qd = q.cuda()
    # one chunk, and chunks that split the stream with a ragged last chunk
    for chunk in (0, 2 * 4099, 2 * 12345):
        got = u32(N.mphf_query_u64_windowed(m, qd, window_bytes=window_bytes, chunk_keys=chunk))
        assert np.array_equal(got, want), f"W={windows} chunk={chunk}: {int((got != want).sum())} mismatches"


@pytest.mark.parametrize("count", [1, 2, 3, 1023, 1025, 2047, 2048, 2049, 4097, 2 * 4096 + 1])
def test_windowed_query_ragged_counts(count):
    """Counts below, at and around the 1024-, 2048- and 4096-key tiles of the passes."""
    N = need_gpu()
    n = 50_000
    ref, blob = oracle_structure(n, 0, slots_override=4096, alpha=0.9)
    m = N.mphf_deserialize(blob)
    q = _query_stream(n)[:count]
    sentinel = 0x7A7A7A7A
    out = torch.full((count + 2,), sentinel, dtype=torch.int32, device="cuda")
    N.mphf_query_u64_windowed(m, q.cuda(), out[:count], window_bytes=1000, chunk_keys=0)
    got = u32(out[:count])
    assert np.array_equal(got, ref.query_u64(W.as_uint64_numpy(q)))
    assert (out[count:].cpu() == sentinel).all(), "wrote past the output"


def test_one_window_is_the_single_pass_and_alignment_is_checked():
    N = need_gpu()
    n = 30_000
    ref, blob = oracle_structure(n, 0, slots_override=2048, alpha=0.9)
    m = N.mphf_deserialize(blob)
    q = _query_stream(n).cuda()
    want = ref.query_u64(W.as_uint64_numpy(q))
    assert np.array_equal(u32(N.mphf_query_u64_windowed(m, q, window_bytes=1 << 40)), want)
    # 8-byte but not 16-byte aligned keys: the single pass accepts them, the windowed path refuses
    buf = torch.empty(q.numel() + 1, dtype=torch.int64, device="cuda")
    buf[1:] = q
    odd = buf[1:]
    assert np.array_equal(u32(N.mphf_query_u64(m, odd)), want)
    with pytest.raises(N.MphfError) as e:
        N.mphf_query_u64_windowed(m, odd, window_bytes=4096)
    assert e.value.code == N.MPHF_ERR_ARG
    with pytest.raises(N.MphfError):
        N.mphf_query_u64_windowed(m, q, window_bytes=4096, chunk_keys=4097)   # odd chunk


def test_windowed_queries_from_two_streams_and_a_growing_scratch():
    """The scratch belongs to the structure: queries from two threads on two
    streams are ordered on the GPU, and a larger chunk grows it."""
    N = need_gpu()
    n = 10**6
    ref, blob = oracle_structure(n, 0)
    m = N.mphf_deserialize(blob)
    q = _query_stream(n).cuda()
    want = ref.query_u64(W.as_uint64_numpy(q))
    outs = [torch.empty(q.numel(), dtype=torch.int32, device="cuda") for _ in range(4)]
    torch.cuda.synchronize()

    def run(i):
        s = torch.cuda.Stream()
        with torch.cuda.stream(s):
            for rep in range(3):
                N.mphf_query_u64_windowed(m, q, outs[i], window_bytes=60_000, chunk_keys=2 * (20_000 + 7000 * i),
                                          stream=s)
        s.synchronize()

    ts = [threading.Thread(target=run, args=(i,)) for i in range(4)]
    for t in ts:
        t.start()
    for t in ts:
        t.join()
    for o in outs:
        assert np.array_equal(u32(o), want)


def test_automatic_path_matches_oracle_on_a_large_batch():
    """mphf_query_u64 takes the windowed path by itself for >= 2^24 keys on a
    pilot array above 72 MiB; a 3e8-key structure has 86 MB of pilots.  The
    structure is built by the library; its serialized bytes are evaluated by
    the oracle on a sample, and the whole output equals the single pass."""
    N = need_gpu()
    n = 3 * 10**8
    keys = W.u64_keys(n, 12, device="cuda")
    m = N.mphf_build(keys)
    info = N.mphf_info(m)
    assert info["P"] * info["B"] > 72 << 20
    q = keys[:1 << 25].contiguous()
    del keys
    torch.cuda.empty_cache()
    auto = N.mphf_query_u64(m, q)
    single = N.mphf_query_u64_windowed(m, q, window_bytes=1 << 40)
    assert torch.equal(auto, single)
    # either side of the 2^24-key threshold of the automatic choice
    for cnt in ((1 << 24) - 1, 1 << 24):
        assert torch.equal(N.mphf_query_u64(m, q[:cnt]), single[:cnt])
    idx = W.uniform_index(200_000, q.numel(), 3).cuda()
    ref = O.OracleMPHF.deserialize(N.mphf_serialize(m))
    assert np.array_equal(u32(auto[idx]), ref.query_u64(W.as_uint64_numpy(q[idx]), threads=16))


@pytest.mark.parametrize("params", [{"remap": O.REMAP_VEC},
                                    {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}],
                         ids=["gamma3", "gamma1"])
def test_phf_wide_and_lookup_take_the_windowed_path_with_the_same_values(params):
    """The PHF query (slots), the 64-bit query and the fused lookup choose the
    windowed path like mphf_query_u64: on a 3e8-key structure and a 2^25-key
    batch each must equal its single-pass result and the oracle.  Both
    structures have two windows; with gamma_1 every last pass computes the
    bucket from the key and the first pass writes no bucket stream, with
    gamma_3 only the lookup's does."""
    N = need_gpu()
    n = 3 * 10**8
    keys = W.u64_keys(n, 13, device="cuda")
    m = N.mphf_build(keys, N.mphf_default_params(**params))
    info = N.mphf_info(m)
    assert info["pilot_bytes"] > 72 << 20 and -(-info["pilot_bytes"] // 100_000_000) <= 2
    q = torch.cat([keys[:(1 << 25) - 1000], W.nonmember_u64_keys(1000, n, 13, device="cuda")]).contiguous()
    del keys
    torch.cuda.empty_cache()
    ref = O.OracleMPHF.deserialize(N.mphf_serialize(m))
    idx = torch.cat([W.uniform_index(100_000, q.numel(), 4), torch.arange(q.numel() - 1000, q.numel())]).cuda()
    qs = W.as_uint64_numpy(q[idx])
    want_vals = ref.query_u64(qs, threads=16)
    # 64-bit values (windowed: 16-byte aligned output)
    wide = N.mphf_query_u64_wide(m, q)
    assert np.array_equal(wide[idx].cpu().numpy().view(np.uint64), want_vals.astype(np.uint64))
    assert torch.equal(wide.to(torch.int32), N.mphf_query_u64_windowed(m, q, window_bytes=1 << 40))
    # slots without the remap
    phf = N.mphf_query_u64_phf(m, q)
    assert np.array_equal(u32(phf[idx]), ref.slots_u64(qs).astype(np.uint32))
    # fused lookup, 4- and 8-byte tables whose entry j names j
    for dtype in (torch.int32, torch.int64):
        table = torch.arange(n, dtype=dtype, device="cuda") ^ 0x5A5A5A5A
        got = N.mphf_lookup_u64(m, q, table)
        assert torch.equal(got, table[wide])
        del table, got
        torch.cuda.empty_cache()

