"""Multi-structure persistent batch kernel against the oracle (bit-exact).

Oracle-built structures of mixed layouts, log-uniform request sizes, 90%
member and 10% non-member keys; every request's output must equal the
oracle's one-by-one evaluation, for every launch shape, with and without
the captured graph, on consecutive runs (both staging sets)."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, u32

pytestmark = pytest.mark.gpu


def make_set(n_mphf=24, nmax=200_000, qmax=20_000, seed=2):
    """Structures with n log-uniform in [1e3, nmax] and requests of log-uniform size."""
    ns = W.log_uniform_int(n_mphf, 1e3, nmax, seed).tolist()
    qs = W.log_uniform_int(n_mphf, 1, qmax, seed + 1).tolist()
    structs, reqs = [], []
    for i, (n, qn) in enumerate(zip(ns, qs)):
        params = {} if i % 3 else {"lam": 3.0, "gamma": O.GAMMA_LINEAR, "remap": O.REMAP_VEC}
        keys = W.u64_keys(n, seed=100 + i)
        ref = O.OracleMPHF.build_u64(W.as_uint64_numpy(keys), **params)
        members = keys[W.uniform_index(qn, n, seed=200 + i)]
        nm = qn // 10
        q = torch.cat([members[: qn - nm], W.nonmember_u64_keys(nm, n, seed=100 + i)])
        structs.append(ref)
        reqs.append(q)
    return structs, reqs


@pytest.fixture(scope="module")
def batch_set():
    need_gpu()
    return make_set()


def run_and_check(N, batch, structs, reqs, extra_bytes=None):
    ms = [N.mphf_deserialize(r.serialize()) for r in structs]
    items, outs = [], []
    for m, q in zip(ms, reqs):
        out = torch.full((q.numel(),), -1, dtype=torch.int32, device="cuda")
        items.append((m, q.cuda(), out))
        outs.append(out)
    if extra_bytes is not None:
        ref_b, data, off = extra_bytes
        mb = N.mphf_deserialize(ref_b.serialize())
        outb = torch.full((off.numel() - 1,), -1, dtype=torch.int32, device="cuda")
        items.append((mb, data.cuda(), off.cuda(), outb))
    arr, keep = N.make_requests(items)
    batch.run(arr, len(items))
    torch.cuda.synchronize()
    for ref, q, out in zip(structs, reqs, outs):
        assert np.array_equal(u32(out), ref.query_u64(W.as_uint64_numpy(q)))
    if extra_bytes is not None:
        assert np.array_equal(u32(outb), ref_b.query_bytes(data.numpy(), off.numpy().astype(np.uint64)))
    return ms, keep


@pytest.mark.parametrize("cfg", [(8, 256, 4, True), (2, 128, 1, True), (16, 512, 2, True), (4, 256, 8, False)])
def test_batch_matches_oracle(batch_set, cfg):
    N = need_gpu()
    structs, reqs = batch_set
    b = N.Batch(64)
    b.set_config(*cfg)
    for _ in range(3):   # consecutive runs use both staging sets
        run_and_check(N, b, structs, reqs)


def test_batch_mixes_u64_and_string_structures(batch_set):
    N = need_gpu()
    structs, reqs = batch_set
    ids = torch.arange(3000)
    data, off = W.strings(ids, seed=9)
    ref_b = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64))
    qd, qo = W.strings(torch.cat([ids[W.permutation(3000, 1)], torch.arange(3000, 3300)]), seed=9)
    b = N.Batch(64)
    run_and_check(N, b, structs[:8], reqs[:8], extra_bytes=(ref_b, qd, qo))


def test_batch_empty_requests_and_capacity(batch_set):
    N = need_gpu()
    structs, _ = batch_set
    m = N.mphf_deserialize(structs[0].serialize())
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    out = torch.empty(0, dtype=torch.int32, device="cuda")
    b = N.Batch(4)
    arr, keep = N.make_requests([(m, empty, out)] * 2)
    b.run(arr, 2)
    arr, keep = N.make_requests([(m, empty, out)] * 5)
    with pytest.raises(N.MphfError) as e:
        b.run(arr, 5)
    assert e.value.code == N.MPHF_ERR_CAPACITY


def test_autotune_picks_a_valid_shape_and_caches_it(batch_set, tmp_path):
    N = need_gpu()
    structs, reqs = batch_set
    ms = [N.mphf_deserialize(r.serialize()) for r in structs]
    items = [(m, q.cuda(), torch.empty(q.numel(), dtype=torch.int32, device="cuda")) for m, q in zip(ms, reqs)]
    arr, keep = N.make_requests(items)
    b = N.Batch(64)
    cache = tmp_path / "tune.jsonl"
    best = b.autotune(arr, len(items), str(cache))
    assert best["keys_per_thread"] in (2, 4, 8, 16) and best["threads"] in (128, 256, 512)
    assert cache.read_text().count("keys_per_thread") == 1
    b2 = N.Batch(64)
    assert b2.autotune(arr, len(items), str(cache)) == best           # read from the cache
    assert cache.read_text().count("keys_per_thread") == 1
    run_and_check(N, b2, structs, reqs)


def test_autotune_ignores_a_shape_cached_by_another_build(batch_set, tmp_path):
    """The cache key holds the library's build time: an entry written by another
    build of the kernel (whose best shape may differ) is not reused."""
    import json
    N = need_gpu()
    structs, reqs = batch_set
    ms = [N.mphf_deserialize(r.serialize()) for r in structs]
    items = [(m, q.cuda(), torch.empty(q.numel(), dtype=torch.int32, device="cuda")) for m, q in zip(ms, reqs)]
    arr, keep = N.make_requests(items)
    cache = tmp_path / "tune.jsonl"
    N.Batch(64).autotune(arr, len(items), str(cache))
    entry = json.loads(cache.read_text().splitlines()[0])
    assert entry["build"]
    planted = dict(entry, build="Jan  1 2000 00:00:00", keys_per_thread=2, threads=128, blocks_per_sm=1)
    cache.write_text(json.dumps(planted) + "\n")
    best = N.Batch(64).autotune(arr, len(items), str(cache))
    lines = cache.read_text().splitlines()
    assert len(lines) == 2 and json.loads(lines[1])["build"] == entry["build"]
    assert (best["keys_per_thread"], best["threads"], best["blocks_per_sm"]) == \
        (json.loads(lines[1])["keys_per_thread"], json.loads(lines[1])["threads"], json.loads(lines[1])["blocks_per_sm"])


def test_batch_refuses_128_bit_string_structures():
    """The batch executor returns 32-bit results through the 64-bit string
    hash only; a structure with the 128-bit hash is refused, not misread."""
    N = need_gpu()
    ids = torch.arange(500)
    data, off = W.strings(ids, seed=10)
    ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), hash128=1)
    m = N.mphf_deserialize(ref.serialize())
    out = torch.full((500,), -1, dtype=torch.int32, device="cuda")
    arr, keep = N.make_requests([(m, data.cuda(), off.cuda(), out)])
    with pytest.raises(N.MphfError) as e:
        N.Batch(4).run(arr, 1)
    assert e.value.code == N.MPHF_ERR_ARG


def test_batch_with_empty_requests_between_others(batch_set):
    """Empty requests own no tile, so several requests start at the same tile
    index; every tile must still go to the non-empty request that owns it."""
    N = need_gpu()
    structs, reqs = batch_set
    ms = [N.mphf_deserialize(r.serialize()) for r in structs]
    empty = torch.empty(0, dtype=torch.int64, device="cuda")
    empty_out = torch.empty(0, dtype=torch.int32, device="cuda")
    items, outs = [(ms[0], empty, empty_out)], []
    for i, (m, q) in enumerate(zip(ms, reqs)):
        out = torch.full((q.numel(),), -1, dtype=torch.int32, device="cuda")
        items.append((m, q.cuda(), out))
        outs.append(out)
        if i % 3 == 1:
            items += [(m, empty, empty_out)] * 2
    items.append((ms[-1], empty, empty_out))
    arr, keep = N.make_requests(items)
    for cfg in [(2, 128, 1, True), (8, 256, 4, True)]:
        b = N.Batch(len(items))
        b.set_config(*cfg)
        for o in outs:
            o.fill_(-1)
        b.run(arr, len(items))
        torch.cuda.synchronize()
        for ref, q, out in zip(structs, reqs, outs):
            assert np.array_equal(u32(out), ref.query_u64(W.as_uint64_numpy(q)))


def test_batch_with_unaligned_keys_and_outputs(batch_set):
    """Full tiles take the paired 16-byte key loads only when a request's keys
    are 16-byte and its outputs 8-byte aligned; views one element into their
    buffers (8-byte aligned keys, 4-byte aligned outputs) take the checked
    per-key path and must give the same values."""
    N = need_gpu()
    structs, reqs = batch_set
    ms = [N.mphf_deserialize(r.serialize()) for r in structs]
    items, outs, keep_bufs = [], [], []
    for i, (m, q) in enumerate(zip(ms, reqs)):
        kbuf = torch.empty(q.numel() + 1, dtype=torch.int64, device="cuda")
        obuf = torch.full((q.numel() + 1,), -1, dtype=torch.int32, device="cuda")
        ks = kbuf[1:] if i % 2 else kbuf[:-1]
        os_ = obuf[1:] if i % 3 else obuf[:-1]
        ks.copy_(q.cuda())
        items.append((m, ks, os_))
        outs.append(os_)
        keep_bufs += [kbuf, obuf]
    arr, keep = N.make_requests(items)
    for cfg in [(4, 512, 4, True), (2, 128, 1, True)]:
        b = N.Batch(len(items))
        b.set_config(*cfg)
        for o in outs:
            o.fill_(-1)
        b.run(arr, len(items))
        torch.cuda.synchronize()
        for ref, q, out in zip(structs, reqs, outs):
            assert np.array_equal(u32(out), ref.query_u64(W.as_uint64_numpy(q)))
