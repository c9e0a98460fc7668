"""Serving loop: continuous batching over resident structures.

Each request's result must equal the oracle's whether it runs alone on an
idle server or mixed with many concurrent requests of other structures
arriving while batches are in flight, also when the HBM budget forces
structures to be evicted and re-admitted."""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, u32

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def fleet():
    need_gpu()
    structs = []
    for i, n in enumerate([3000, 40_000, 250_000, 1_200_000]):
        keys = W.u64_keys(n, seed=300 + i)
        structs.append(("u64", O.OracleMPHF.build_u64(W.as_uint64_numpy(keys), threads=8), keys))
    ids = torch.arange(20_000)
    data, off = W.strings(ids, seed=11)
    structs.append(("bytes", O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=8), ids))
    return structs


def make_request(kind, ref, keys, count, seed):
    """A request of `count` keys: 90% members, 10% non-members; returns the
    device inputs and the oracle's expected output."""
    if kind == "u64":
        n = keys.numel()
        nm = count // 10
        q = torch.cat([keys[W.uniform_index(count - nm, n, seed)], W.nonmember_u64_keys(nm, n, seed)])
        return (q.cuda(), None), ref.query_u64(W.as_uint64_numpy(q))
    ids = torch.cat([keys[W.uniform_index(count - count // 10, keys.numel(), seed)],
                     keys.numel() + W.uniform_index(count // 10, 10_000, seed)])
    d, o = W.strings(ids, seed=11)
    return (d.cuda(), o.cuda()), ref.query_bytes(d.numpy(), o.numpy().astype(np.uint64))


def test_result_is_the_same_alone_and_in_the_mix(fleet):
    N = need_gpu()
    srv = N.Server(slots=3, max_batch_requests=64, max_batch_keys=1 << 20)
    sids = [srv.add(ref.serialize()) for _, ref, _ in fleet]
    probe_kind, probe_ref, probe_keys = fleet[2]
    (pk, po), want = make_request(probe_kind, probe_ref, probe_keys, 50_000, seed=1)
    out_alone = torch.full((50_000,), -1, dtype=torch.int32, device="cuda")
    assert srv.wait(srv.submit(N.Server.request(sids[2], pk, out_alone))) == N.MPHF_OK
    assert np.array_equal(u32(out_alone), want)

    # The mix: 300 requests of every structure, log-uniform sizes, Poisson
    # arrivals, with the probe request in the middle.
    sizes = W.log_uniform_int(300, 1, 200_000, seed=7).tolist()
    gaps = -np.log(1.0 - np.random.default_rng(3).random(300)) * 20.0     # mean 20 us
    reqs, expect, outs, keep = [], [], [], []
    for r, cnt in enumerate(sizes):
        k = r % len(fleet)
        kind, ref, keys = fleet[k]
        if r == 150:
            k, kind, ref, keys, cnt = 2, probe_kind, probe_ref, probe_keys, 50_000
            (dk, do), exp = (pk, po), want
        else:
            (dk, do), exp = make_request(kind, ref, keys, cnt, seed=1000 + r)
        out = torch.full((cnt,), -1, dtype=torch.int32, device="cuda")
        reqs.append(N.Server.request(sids[k], dk, out, do))
        expect.append(exp)
        outs.append(out)
        keep.append((dk, do))
    torch.cuda.synchronize()
    tickets = srv.replay(reqs, np.cumsum(gaps))
    for t in tickets:
        assert srv.wait(t) == N.MPHF_OK
    for out, exp in zip(outs, expect):
        assert np.array_equal(u32(out), exp)
    assert np.array_equal(u32(outs[150]), u32(out_alone))
    st = srv.stats()
    assert st["requests"] == 301 and st["p50_us"] <= st["p99_us"] <= st["max_us"]
    assert st["batches"] < 301          # requests were coalesced
    srv.close()


def test_admission_by_hbm_budget_evicts_and_readmits(fleet):
    N = need_gpu()
    blobs = [ref.serialize() for _, ref, _ in fleet]
    sizes = [N.mphf_info(N.mphf_deserialize(b))["pilot_bytes"] + N.mphf_info(N.mphf_deserialize(b))["remap_bytes"]
             for b in blobs]
    budget = max(sizes) + 4096            # room for about one structure at a time
    srv = N.Server(hbm_budget_bytes=budget, slots=2)
    sids = [srv.add(b) for b in blobs]
    reqs, expect, outs, keep = [], [], [], []
    for r in range(40):
        k = (r * 3) % len(fleet)
        kind, ref, keys = fleet[k]
        (dk, do), exp = make_request(kind, ref, keys, 5000, seed=5000 + r)
        out = torch.full((5000,), -1, dtype=torch.int32, device="cuda")
        reqs.append(N.Server.request(sids[k], dk, out, do))
        expect.append(exp)
        outs.append(out)
        keep.append((dk, do))
    tickets = srv.replay(reqs, [10.0 * i for i in range(40)])
    for t in tickets:
        assert srv.wait(t) == N.MPHF_OK
    for out, exp in zip(outs, expect):
        assert np.array_equal(u32(out), exp)
    st = srv.stats()
    assert st["evictions"] > 0 and st["admissions"] > len(fleet)
    assert st["resident_bytes"] <= budget
    srv.remove(sids[0])
    with pytest.raises(N.MphfError):
        srv.submit(N.Server.request(sids[0], keep[0][0], outs[0]))
    srv.close()


def test_server_errors(fleet):
    N = need_gpu()
    srv = N.Server(hbm_budget_bytes=1000)
    with pytest.raises(N.MphfError) as e:
        srv.add(fleet[3][1].serialize())
    assert e.value.code == N.MPHF_ERR_CAPACITY
    with pytest.raises(N.MphfError) as e:
        srv.add(b"garbage" * 40)
    assert e.value.code == N.MPHF_ERR_FORMAT
    with pytest.raises(N.MphfError) as e:
        srv.submit(N.Server.request(7, torch.empty(0, dtype=torch.int64), torch.empty(0, dtype=torch.int32)))
    assert e.value.code == N.MPHF_ERR_ARG
    srv.drain()
    srv.close()
