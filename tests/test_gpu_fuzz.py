"""Seeded random layouts, bit-exact against the oracle.

Each case draws n, lambda, alpha, gamma, the remap kind, the key kind
(u64, strings, strings with the 128-bit hash) and sometimes a forced slot
count (power of two or not, hence both reduce modes), builds the structure
with the oracle and checks every query path of the library on it: 32-bit
and 64-bit results, members and non-members.  The library's own builder
then builds the same key set under the same parameters: that structure must
be a bijection (Sec. 3.2), and the oracle, loading its serialized bytes,
must give the GPU's values on members and non-members alike."""
from __future__ import annotations

import random

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests.gpu_common import need_gpu, oracle_values_of, u32

pytestmark = pytest.mark.gpu


def draw(case: int) -> dict:
    r = random.Random(1000 + case)
    n = int(10 ** r.uniform(0.5, 5.3))
    p = {"lam": r.choice([3.0, 3.5, 4.0]), "alpha": r.choice([0.85, 0.9, 0.95, 0.99]),
         "gamma": r.choice([O.GAMMA_LINEAR, O.GAMMA_CUBIC]), "remap": r.choice([O.REMAP_CLEF, O.REMAP_VEC]),
         "seed": r.randrange(1 << 32)}
    if n >= 2000 and r.random() < 0.6:   # many parts, either reduce mode
        p["slots_override"] = r.choice([1024, 2048, 4096, 1500, 3001])
    kind = r.choice(["u64", "u64", "bytes", "bytes128"])
    return {"n": n, "params": p, "kind": kind, "key_seed": r.randrange(1 << 16)}


CASES = [draw(i) for i in range(24)]


def ids(c):
    p = c["params"]
    return f"{c['kind']}-n{c['n']}-g{p['gamma']}-r{p['remap']}-S{p.get('slots_override', 0)}"


@pytest.mark.parametrize("case", CASES, ids=[ids(c) for c in CASES])
def test_random_layout_matches_oracle(case):
    N = need_gpu()
    n, p, kind, ks = case["n"], case["params"], case["kind"], case["key_seed"]
    if kind == "u64":
        keys = W.u64_keys(n, ks)
        ref = O.OracleMPHF.build_u64(W.as_uint64_numpy(keys), threads=8, **p)
        m = N.mphf_deserialize(ref.serialize())
        q = torch.cat([keys[W.permutation(n, ks + 1)], W.nonmember_u64_keys(n // 3 + 5, n, ks)])
        want = ref.query_u64(W.as_uint64_numpy(q))
        assert np.array_equal(u32(N.mphf_query_u64(m, q.cuda())), want)
        assert np.array_equal(N.mphf_query_u64_wide(m, q.cuda()).cpu().numpy().view(np.uint64), want)
        gpu = N.mphf_build(keys.cuda(), N.mphf_default_params(**p))
        got = u32(N.mphf_query_u64(gpu, keys.cuda()))
        assert np.array_equal(u32(N.mphf_query_u64(gpu, q.cuda())), oracle_values_of(N, gpu, keys=q))
    else:
        h128 = 1 if kind == "bytes128" else 0
        data, off = W.strings(torch.arange(n), seed=ks)
        ref = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), threads=8, hash128=h128, **p)
        m = N.mphf_deserialize(ref.serialize())
        qd, qo = W.strings(torch.cat([torch.arange(n)[W.permutation(n, ks + 1)], torch.arange(n, n + n // 3 + 5)]),
                           seed=ks)
        want = ref.query_bytes(qd.numpy(), qo.numpy().astype(np.uint64))
        assert np.array_equal(u32(N.mphf_query_bytes(m, qd.cuda(), qo.cuda())), want)
        assert np.array_equal(N.mphf_query_bytes_wide(m, qd.cuda(), qo.cuda()).cpu().numpy().view(np.uint64), want)
        gpu = N.mphf_build(data.cuda(), N.mphf_default_params(hash128=h128, **p), offsets=off.cuda())
        got = u32(N.mphf_query_bytes(gpu, data.cuda(), off.cuda()))
        assert np.array_equal(u32(N.mphf_query_bytes(gpu, qd.cuda(), qo.cuda())),
                              oracle_values_of(N, gpu, data=qd, offsets=qo))
    assert np.array_equal(np.sort(got), np.arange(n, dtype=np.uint32))
