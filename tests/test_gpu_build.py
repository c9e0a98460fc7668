"""The library's own GPU builder: every structure it builds must be a
bijection onto [0, n) for its keys, whatever the layout (Sec. 3.2), and the
GPU's values must equal the oracle's evaluation of the same serialized
structure; its errors follow the same rules as the oracle's."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, oracle_values_of, u32

pytestmark = pytest.mark.gpu


def check_bijection(N, m, keys_dev, n):
    """A bijection onto [0, n), and element-wise the oracle's values for the
    same serialized structure."""
    got = u32(N.mphf_query_u64(m, keys_dev))
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32))
    assert np.array_equal(got, oracle_values_of(N, m, keys=keys_dev))


def check_strings(N, m, data, off, n):
    got = u32(N.mphf_query_bytes(m, data, off))
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32))
    assert np.array_equal(got, oracle_values_of(N, m, data=data, offsets=off))


BUILD_CASES = [
    (1, {}), (2, {}), (23, {}), (1000, {}), (20_000, {}), (200_000, {}),
    (10**6, {}), (10**6, {"lam": 3.0, "gamma": 1, "remap": 1}), (10**6, {"lam": 4.0}),
    (30_000, {"slots_override": 2048, "alpha": 0.9}),
    (30_000, {"slots_override": 3001, "alpha": 0.9}),
    (5 * 10**6, {}),
]


@pytest.mark.parametrize("n,params", BUILD_CASES)
def test_gpu_build_is_bijective(n, params):
    N = need_gpu()
    keys = W.u64_keys(n, 1).cuda()
    m = N.mphf_build(keys, N.mphf_default_params(**params))
    info = N.mphf_info(m)
    assert info["n"] == n
    check_bijection(N, m, keys, n)
    other = W.nonmember_u64_keys(1000, n, 1).cuda()
    vals = u32(N.mphf_query_u64(m, other))
    assert vals.max() < n
    assert np.array_equal(vals, oracle_values_of(N, m, keys=other))
    # The serialized structure reloads to the same function.
    m2 = N.mphf_deserialize(N.mphf_serialize(m))
    assert np.array_equal(u32(N.mphf_query_u64(m2, keys)), u32(N.mphf_query_u64(m, keys)))


@pytest.mark.parametrize("n", [50_000, 3 * 10**6])
def test_gpu_build_is_deterministic(n):
    """The same keys and parameters give the same structure, byte for byte."""
    N = need_gpu()
    keys = W.u64_keys(n, 8).cuda()
    a = N.mphf_serialize(N.mphf_build(keys))
    b = N.mphf_serialize(N.mphf_build(keys))
    assert a == b


def test_gpu_build_remap_invariants():
    """Keys mapping to slots >= n go, in slot order, to the free slots < n (Sec. 3.4)."""
    N = need_gpu()
    n = 10**6
    keys = W.u64_keys(n, 2).cuda()
    m = N.mphf_build(keys)
    slots = u32(N.mphf_query_u64_phf(m, keys)).astype(np.int64)
    final = u32(N.mphf_query_u64(m, keys)).astype(np.int64)
    assert len(np.unique(slots)) == n
    assert np.array_equal(final, oracle_values_of(N, m, keys=keys).astype(np.int64))
    hi = slots >= n
    order = np.argsort(slots[hi])
    taken = np.zeros(n, bool)
    taken[slots[~hi]] = True
    free = np.flatnonzero(~taken)
    assert np.array_equal(final[hi][order], free)
    assert np.array_equal(final[~hi], slots[~hi])


def test_gpu_build_duplicates_rejected():
    N = need_gpu()
    keys = W.u64_keys(5000, 0)
    keys[77] = keys[4000]
    with pytest.raises(N.MphfError) as e:
        N.mphf_build(keys.cuda())
    assert e.value.code == N.MPHF_ERR_DUP_KEYS


def test_gpu_build_eviction_cap():
    """evict_mult = 0 forbids eviction; the default cap of 10 S lets it build."""
    N = need_gpu()
    keys = W.u64_keys(200_000, 4).cuda()
    m = N.mphf_build(keys, N.mphf_default_params(max_reseeds=0))
    assert N.mphf_info(m)["evictions"] > 0
    check_bijection(N, m, keys, 200_000)
    with pytest.raises(N.MphfError) as e:
        N.mphf_build(keys, N.mphf_default_params(max_reseeds=0, evict_mult=0))
    assert e.value.code == N.MPHF_ERR_BUILD_FAILED
    assert "mixer" in str(e.value)   # the message names the remedy for structured keys


@pytest.mark.parametrize("n", [1, 100, 50_000])
def test_gpu_build_strings_bijective(n):
    N = need_gpu()
    data, off = W.strings(torch.arange(n), seed=6)
    m = N.mphf_build(data.cuda(), offsets=off.cuda())
    check_strings(N, m, data.cuda(), off.cuda(), n)


def test_gpu_build_duplicate_strings_rejected():
    N = need_gpu()
    data, off = W.strings(torch.tensor([0, 1, 2, 3, 1]), seed=6)
    with pytest.raises(N.MphfError) as e:
        N.mphf_build(data.cuda(), N.mphf_default_params(max_reseeds=2), offsets=off.cuda())
    assert e.value.code == N.MPHF_ERR_DUP_KEYS


# (n, shard_keys): 1e6 keys are P = 4 parts, 3e6 are 6, 2e7 are 39; the shard
# sizes give one part per shard, uneven shards, and many shards.
SHARD_CASES = [(10**6, 300_000), (10**6, 600_000), (3 * 10**6, 1_400_000), (2 * 10**7, 3_000_000)]


@pytest.mark.parametrize("n,shard_keys", SHARD_CASES)
def test_sharded_build_is_identical(n, shard_keys):
    """In-memory sharding by part ranges (Appendix B, Sharding) changes only
    how the build walks the keys: the structure is the same, byte for byte."""
    N = need_gpu()
    keys = W.u64_keys(n, 9).cuda()
    whole = N.mphf_serialize(N.mphf_build(keys))
    m = N.mphf_build(keys, N.mphf_default_params(shard_keys=shard_keys))
    assert N.mphf_serialize(m) == whole
    check_bijection(N, m, keys, n)


def test_sharded_string_build_is_identical():
    N = need_gpu()
    n = 300_000
    data, off = W.strings(torch.arange(n), seed=7)
    data, off = data.cuda(), off.cuda()
    whole = N.mphf_serialize(N.mphf_build(data, offsets=off))
    m = N.mphf_build(data, N.mphf_default_params(shard_keys=40_000), offsets=off)   # P = 3: three shards
    assert N.mphf_serialize(m) == whole
    check_strings(N, m, data, off, n)


@pytest.mark.parametrize("n", [1, 1000, 300_000])
def test_gpu_build_with_128_bit_string_hash(n):
    """The GPU builder with the 128-bit string hash (forced here; automatic
    past 2^32 keys): a bijection, flagged in the header, and the same bytes
    when built in shards."""
    N = need_gpu()
    data, off = W.strings(torch.arange(n), seed=14)
    data, off = data.cuda(), off.cuda()
    m = N.mphf_build(data, N.mphf_default_params(hash128=1), offsets=off)
    blob = N.mphf_serialize(m)
    assert int.from_bytes(blob[28:32], "little") == 1
    check_strings(N, m, data, off, n)
    if n >= 300_000:   # P = 3: three shards
        sharded = N.mphf_build(data, N.mphf_default_params(hash128=1, shard_keys=40_000), offsets=off)
        assert N.mphf_serialize(sharded) == blob


def test_gpu_build_128_bit_duplicate_strings_rejected():
    N = need_gpu()
    data, off = W.strings(torch.tensor([0, 1, 2, 3, 1]), seed=6)
    with pytest.raises(N.MphfError) as e:
        N.mphf_build(data.cuda(), N.mphf_default_params(max_reseeds=2, hash128=1), offsets=off.cuda())
    assert e.value.code == N.MPHF_ERR_DUP_KEYS


def test_concurrent_builds_from_threads_match_sequential_builds():
    """Builds from several host threads, each on its own stream, overlap on
    the GPU (stream-ordered temporaries, one fixed shared-memory limit) and
    give the same bytes as one build at a time."""
    from concurrent.futures import ThreadPoolExecutor
    N = need_gpu()
    ns = [1000, 50_000, 300_000, 2_000_000, 7_000, 900_000, 120_000, 4_000_000]
    keys = [W.u64_keys(n, 40 + i).cuda() for i, n in enumerate(ns)]
    data, off = W.strings(torch.arange(200_000), seed=41)
    data, off = data.cuda(), off.cuda()
    want = [N.mphf_serialize(N.mphf_build(k)) for k in keys] + [N.mphf_serialize(N.mphf_build(data, offsets=off))]

    def build(i):
        stream = torch.cuda.Stream()
        with torch.cuda.stream(stream):
            if i < len(keys):
                m = N.mphf_build(keys[i], stream=stream)
            else:
                m = N.mphf_build(data, offsets=off, stream=stream)
        return N.mphf_serialize(m)

    with ThreadPoolExecutor(max_workers=len(want)) as pool:
        got = list(pool.map(build, range(len(want))))
    assert got == want


def test_build_reports_its_phase_times():
    """mphf_info splits the device time of a build into hashing and sorting,
    the pilot search and the remap; the three fit inside the whole."""
    N = need_gpu()
    m = N.mphf_build(W.u64_keys(2_000_000, 11).cuda())
    info = N.mphf_info(m)
    phases = (info["build_hash_sort_ms"], info["build_search_ms"], info["build_remap_ms"])
    assert all(t > 0 for t in phases)
    assert sum(phases) <= info["build_ms"] * 1.001
    loaded = N.mphf_info(N.mphf_deserialize(N.mphf_serialize(m)))
    assert loaded["build_ms"] == 0 and loaded["build_search_ms"] == 0


@pytest.mark.parametrize("t", [8, 20])
def test_gpu_build_small_layout_keys_with_trailing_zeros(t):
    """Keys k 2^t in an x mod S layout (n = 1000): the odd S keeps every slot reachable, so the
    GPU build succeeds and is a bijection, and it equals the oracle's layout."""
    N = need_gpu()
    n = 1000
    keys = (torch.arange(1, n + 1, dtype=torch.int64) << t).cuda()
    m = N.mphf_build(keys)
    info = N.mphf_info(m)
    assert info["S"] % 2 == 1
    L = O.layout_for(n)
    assert (info["P"], info["S"], info["B"]) == (L.P, L.S, L.B)
    check_bijection(N, m, keys, n)
