"""GPU query kernels against the oracle, element by element (bit-exact).

Every structure here is built by the oracle and loaded into the library with
mphf_deserialize; the GPU result for each key must equal the oracle's
one-by-one evaluation (Sec. 3.1 Eq. slot, Sec. 3.4 remap)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, oracle_structure, u32

pytestmark = pytest.mark.gpu

# (n, params): layouts POW2 / MOD, gamma_1 / gamma_3, CacheLineEF / Vec,
# one part and many parts.
CASES = [
    (1, {}),
    (23, {}),
    (1000, {}),
    (4097, {"gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),
    (30_000, {"slots_override": 2048, "alpha": 0.9}),                       # 17 parts, POW2
    (30_000, {"slots_override": 3001, "alpha": 0.9}),                       # 12 parts, x mod S
    (50_000, {"slots_override": 4096, "alpha": 0.95, "gamma": O.GAMMA_LINEAR}),
    (200_000, {}),                                                          # MOD layout
    (10**6, {}),                                                            # P=4, S=2^18 (1e6 config)
    (10**6, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),   # Fast
    (10**6, {"lam": 4.0}),                                                  # Compact
    (3 * 10**6, {"seed": 5}),
]


def ids(c):
    n, p = c
    return f"n{n}-" + "-".join(f"{k}{v}" for k, v in sorted(p.items()))


@pytest.mark.parametrize("case", CASES, ids=[ids(c) for c in CASES])
def test_query_u64_matches_oracle(case):
    N = need_gpu()
    n, params = case
    ref, blob = oracle_structure(n, 0, **params)
    m = N.mphf_deserialize(blob)
    info = N.mphf_info(m)
    assert info["n"] == n and info["P"] == ref.layout.P
    keys = W.u64_keys(n, 0)
    q = torch.cat([keys[W.permutation(n, 1)], W.nonmember_u64_keys(max(n // 4, 17), n, 0)])
    got = u32(N.mphf_query_u64(m, q.cuda()))
    want = ref.query_u64(W.as_uint64_numpy(q))
    assert np.array_equal(got, want), f"{int((got != want).sum())} mismatches"
    assert np.array_equal(np.sort(got[:n]), np.arange(n, dtype=np.uint32))
    assert got.max() < n


@pytest.mark.parametrize("case", CASES[2:10], ids=[ids(c) for c in CASES[2:10]])
def test_wide_query_matches_oracle(case):
    """The 64-bit-result query (needed past 2^32 keys) gives the same values."""
    N = need_gpu()
    n, params = case
    ref, blob = oracle_structure(n, 0, **params)
    m = N.mphf_deserialize(blob)
    q = torch.cat([W.u64_keys(n, 0)[W.permutation(n, 1)], W.nonmember_u64_keys(max(n // 4, 17), n, 0)])
    got = N.mphf_query_u64_wide(m, q.cuda()).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, ref.query_u64(W.as_uint64_numpy(q)))


@pytest.mark.parametrize("n,params", [(5000, {}), (100_000, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC})])
def test_wide_bytes_query_matches_oracle(n, params):
    N = need_gpu()
    ids_ = torch.arange(n)
    data, off = W.strings(ids_, seed=3)
    ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=8, **params)
    m = N.mphf_deserialize(ref.serialize())
    qd, qo = W.strings(torch.cat([ids_[W.permutation(n, 1)], torch.arange(n, n + n // 4)]), seed=3)
    got = N.mphf_query_bytes_wide(m, qd.cuda(), qo.cuda()).cpu().numpy().view(np.uint64)
    assert np.array_equal(got, ref.query_bytes(qd.numpy(), qo.numpy().astype(np.uint64)))


@pytest.mark.parametrize("case", CASES[4:9], ids=[ids(c) for c in CASES[4:9]])
def test_phf_query_matches_oracle_slots(case):
    N = need_gpu()
    n, params = case
    ref, blob = oracle_structure(n, 0, **params)
    m = N.mphf_deserialize(blob)
    keys = W.u64_keys(n, 0)
    got = u32(N.mphf_query_u64_phf(m, keys.cuda())).astype(np.uint64)
    assert np.array_equal(got, ref.slots_u64(W.as_uint64_numpy(keys)))


@pytest.mark.parametrize("count", [0, 1, 2, 31, 2047, 2048, 2049, 4095, 10_001])
@pytest.mark.parametrize("offset", [0, 1])
def test_ragged_sizes_and_alignment(count, offset):
    """Tails of a tile, and keys not 16-byte aligned (the scalar path)."""
    N = need_gpu()
    n = 100_000
    ref, blob = oracle_structure(n)
    m = N.mphf_deserialize(blob)
    buf = torch.cat([W.u64_keys(1, 99), W.u64_keys(n, 0)[:count + 1]]).cuda()
    q = buf[offset: offset + count]
    out_buf = torch.full((count + 2,), -1, dtype=torch.int32, device="cuda")
    out = out_buf[offset: offset + count]
    if count:
        N.mphf_query_u64(m, q, out)
    torch.cuda.synchronize()
    got = u32(out)
    want = ref.query_u64(W.as_uint64_numpy(q.cpu()))
    assert np.array_equal(got, want)
    ob = u32(out_buf)
    assert ob[offset + count] == 0xFFFFFFFF and (offset == 0 or ob[0] == 0xFFFFFFFF)  # nothing written outside


def test_host_buffer_query_matches_device_query():
    N = need_gpu()
    n = 10**6
    ref, blob = oracle_structure(n)
    m = N.mphf_deserialize(blob)
    q = W.u64_keys(n, 0)[W.permutation(n, 3)]
    qh = torch.empty_like(q).pin_memory()
    qh.copy_(q)
    # Several staging chunks plus a ragged last one.
    big = torch.cat([qh] * 40 + [qh[:12345]]).pin_memory()
    out = N.mphf_query_u64_host(m, big)
    want = ref.query_u64(W.as_uint64_numpy(q))
    got = out.numpy().view(np.uint32)
    for i in range(40):
        assert np.array_equal(got[i * n:(i + 1) * n], want)
    assert np.array_equal(got[40 * n:], want[:12345])


def test_host_query_from_pageable_memory():
    """Pageable host buffers take the staged copy path."""
    N = need_gpu()
    n = 300_000
    ref, blob = oracle_structure(n)
    m = N.mphf_deserialize(blob)
    q = W.u64_keys(n, 0)[W.permutation(n, 4)]
    out = N.mphf_query_u64_host(m, q.clone())
    assert np.array_equal(out.numpy().view(np.uint32), ref.query_u64(W.as_uint64_numpy(q)))


def test_serialize_round_trip_is_byte_exact():
    N = need_gpu()
    for n, params in [(1000, {}), (30_000, {"slots_override": 3001, "alpha": 0.9}),
                      (10**6, {"remap": O.REMAP_VEC})]:
        ref, blob = oracle_structure(n, 0, **params)
        m = N.mphf_deserialize(blob)
        assert N.mphf_serialize(m) == blob


def test_query_rejects_wrong_key_kind():
    N = need_gpu()
    ids_ = torch.arange(100)
    data, off = W.strings(ids_, seed=0)
    ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64))
    m = N.mphf_deserialize(ref.serialize())
    with pytest.raises(N.MphfError) as e:
        N.mphf_query_u64(m, W.u64_keys(10).cuda())
    assert e.value.code == N.MPHF_ERR_ARG


@pytest.mark.parametrize("n,params", [(1, {}), (37, {}), (5000, {}), (100_000, {}),
                                      (300_000, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC})])
def test_query_bytes_matches_oracle(n, params):
    N = need_gpu()
    ids_ = torch.arange(n)
    data, off = W.strings(ids_, seed=3)
    ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=8, **params)
    m = N.mphf_deserialize(ref.serialize())
    perm = W.permutation(n, 1)
    extra = torch.arange(n, n + max(n // 4, 5))          # non-members: other strings
    qd, qo = W.strings(torch.cat([ids_[perm], extra]), seed=3)
    got = u32(N.mphf_query_bytes(m, qd.cuda(), qo.cuda()))
    want = ref.query_bytes(qd.numpy(), qo.numpy().astype(np.uint64))
    assert np.array_equal(got, want), f"{int((got != want).sum())} mismatches"
    assert np.array_equal(np.sort(got[:n]), np.arange(n, dtype=np.uint32))


def test_query_bytes_long_and_empty_strings():
    """Strings outside the 16..64 mix: empty, and long ones that miss the stage."""
    N = need_gpu()
    lens = [0, 1, 7, 8, 9, 300, 5000, 15, 16, 17] * 40
    rng = np.random.default_rng(0)
    pieces = [rng.integers(0, 256, size=l, dtype=np.uint8) for l in lens]
    for i, p in enumerate(pieces):   # make every string distinct
        if len(p) >= 2:
            p[:2] = [i & 0xFF, i >> 8]
    keep = [i for i, l in enumerate(lens) if l >= 2] + [0]
    pieces = [pieces[i] for i in keep]
    off = np.zeros(len(pieces) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(p) for p in pieces])
    data = np.concatenate(pieces)
    ref = O.OracleMPHF.build_bytes(data, off)
    m = N.mphf_deserialize(ref.serialize())
    got = u32(N.mphf_query_bytes(m, torch.from_numpy(data).cuda(),
                                 torch.from_numpy(off.view(np.int64)).cuda()))
    assert np.array_equal(got, ref.query_bytes(data, off))


def test_query_bytes_mixed_lengths_and_unstaged_blocks():
    """Lengths 0..200 B (every word-count bin, including the > 14 words one),
    a few 3000-B strings that push their 256-string block off the shared-memory
    stage, and a ragged last block."""
    N = need_gpu()
    rng = np.random.default_rng(4)
    n = 5000 + 77
    lens = rng.integers(0, 201, size=n)
    lens[rng.choice(n, size=6, replace=False)] = 3000
    pieces = []
    for i, l in enumerate(lens):
        p = rng.integers(0, 256, size=int(l), dtype=np.uint8)
        if l >= 3:   # distinct strings: the index in the first bytes
            p[:3] = [i & 0xFF, (i >> 8) & 0xFF, 0x7F]
        pieces.append(p)
    keep = [i for i, l in enumerate(lens) if l >= 3] + [int(np.argmin(lens))]
    pieces = [pieces[i] for i in keep]
    off = np.zeros(len(pieces) + 1, dtype=np.uint64)
    off[1:] = np.cumsum([len(p) for p in pieces])
    data = np.concatenate(pieces)
    ref = O.OracleMPHF.build_bytes(data, off)
    m = N.mphf_deserialize(ref.serialize())
    got = u32(N.mphf_query_bytes(m, torch.from_numpy(data).cuda(),
                                 torch.from_numpy(off.view(np.int64)).cuda()))
    assert np.array_equal(got, ref.query_bytes(data, off))
    assert np.array_equal(np.sort(got), np.arange(len(pieces), dtype=np.uint32))


def test_gather_probe_reads_the_table():
    N = need_gpu()
    keys = W.u64_keys(5000, 7)
    table = (torch.arange(1 << 20) % 251).to(torch.uint8)
    out = torch.empty(5000, dtype=torch.int32, device="cuda")
    N.mphf_gather_probe(keys.cuda(), table.cuda(), out)
    k = W.as_uint64_numpy(keys).astype(object)
    idx = [((int(x) * 0x9E3779B97F4A7C15 % (1 << 64)) * (1 << 20)) >> 64 for x in k]
    assert np.array_equal(u32(out), table.numpy()[idx].astype(np.uint32))


@pytest.mark.parametrize("n,params", [(37, {}), (5000, {}), (100_000, {}),
                                      (60_000, {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}),
                                      (30_000, {"slots_override": 2048, "alpha": 0.9})])   # 17 parts
def test_query_bytes_128_bit_hash_matches_oracle(n, params):
    """Structures whose strings use the 128-bit hash (high half: part and
    bucket; low half: slot; Sec. 3.1), built by the oracle: the 32- and
    64-bit-result queries give the oracle's values."""
    N = need_gpu()
    ids_ = torch.arange(n)
    data, off = W.strings(ids_, seed=13)
    ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=8, hash128=1, **params)
    blob = ref.serialize()
    assert int.from_bytes(blob[28:32], "little") == 1
    m = N.mphf_deserialize(blob)
    qd, qo = W.strings(torch.cat([ids_[W.permutation(n, 1)], torch.arange(n, n + n // 4 + 3)]), seed=13)
    want = ref.query_bytes(qd.numpy(), qo.numpy().astype(np.uint64))
    got = u32(N.mphf_query_bytes(m, qd.cuda(), qo.cuda()))
    assert np.array_equal(got, want), f"{int((got != want).sum())} mismatches"
    wide = N.mphf_query_bytes_wide(m, qd.cuda(), qo.cuda()).cpu().numpy().view(np.uint64)
    assert np.array_equal(wide, want)


def test_l2_fetch_granularity_hint_leaves_results_unchanged():
    N = need_gpu()
    n = 200_000
    ref, blob = oracle_structure(n, 0)
    m = N.mphf_deserialize(blob)
    q = W.u64_keys(n, 0)[W.permutation(n, 1)]
    want = ref.query_u64(W.as_uint64_numpy(q))
    before = N.mphf_set_l2_fetch_granularity(128)
    try:
        assert 0 <= before <= 128
        assert N.mphf_set_l2_fetch_granularity(128) in (128, 64, 32, 0)   # read back, maybe clamped
        assert np.array_equal(u32(N.mphf_query_u64(m, q.cuda())), want)
    finally:
        N.mphf_set_l2_fetch_granularity(before)
    assert np.array_equal(u32(N.mphf_query_u64(m, q.cuda())), want)
