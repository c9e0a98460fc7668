"""The oracle's query against a second, independent restatement of the paper.

tests/bigint_ptrhash.py evaluates a serialized structure with Python's
unbounded integers, reading the header, pilots and remap payload from the
bytes itself (Sec. 3.1 Eq. partbucket, Eq. hp, Eq. slot; Sec. 3.3 gamma;
Sec. 3.4 remap and CacheLineEF lookup).  Here every layout the oracle can
produce is built by the oracle, and its one-by-one queries must equal the
restatement key by key, for members and non-members.  This pins the parts
of the oracle that bijection and invariants cannot: the factor C in the
pilot hash, the xor of h and hp, the high half taken by the power-of-two
reduce, and the CacheLineEF decode with a bit-scan select.
"""
from __future__ import annotations

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W
from tests import bigint_ptrhash as R

U64_CASES = {
    # name: (n, key seed, oracle build parameters)
    "single part, x mod S, CacheLineEF": (5000, 21, {}),
    "single part, Fast (gamma_1, lambda 3.0, Vec)": (3000, 22, {"lam": 3.0, "gamma": O.GAMMA_LINEAR,
                                                               "remap": O.REMAP_VEC}),
    "17 parts, power-of-two S, CacheLineEF": (30000, 23, {"slots_override": 2048, "alpha": 0.9}),
    "20 parts, gamma_1, Vec": (20000, 24, {"slots_override": 1024, "alpha": 0.9, "gamma": O.GAMMA_LINEAR,
                                           "remap": O.REMAP_VEC}),
    "11 parts, x mod S": (30000, 25, {"slots_override": 3001, "alpha": 0.9}),
    "Compact (lambda 4.0), seed 7": (4000, 26, {"lam": 4.0, "seed": 7}),
    "n = 1e6, the rule's power-of-two layout": (1_000_000, 0, {"threads": 8}),
}


def _sample(n: int, k: int, seed: int) -> np.ndarray:
    if n <= k:
        return np.arange(n)
    return W.uniform_index(k, n, seed).numpy()


@pytest.mark.parametrize("name", sorted(U64_CASES))
def test_u64_query_equals_the_big_integer_restatement(name):
    n, seed, params = U64_CASES[name]
    keys = W.as_uint64_numpy(W.u64_keys(n, seed))
    m = O.OracleMPHF.build_u64(keys, **params)
    st = R.parse(m.serialize())
    assert st.n == n and st.key_kind == 0
    members = keys[_sample(n, 3000, seed)]
    others = W.as_uint64_numpy(W.nonmember_u64_keys(1000, n, seed))
    q = np.concatenate([members, others])
    got = m.query_u64(q)
    slots = m.slots_u64(q)
    remapped = 0
    for k, g, s in zip(q.tolist(), got.tolist(), slots.tolist()):
        h = (st.C * k) % R.M
        want_slot = R.slot(st, h, h)
        assert s == want_slot, f"{name}: slot of key {k:#x}"
        assert g == R.value_of_hash(st, h, h), f"{name}: value of key {k:#x}"
        remapped += want_slot >= n
    if st.P * st.S > n:
        assert remapped > 0, "the sample must reach the remap table"


STRING_CASES = {
    "64-bit hash, single part": (8000, 31, {}),
    "64-bit hash, 17 parts": (30000, 32, {"slots_override": 2048, "alpha": 0.9}),
    "128-bit hash, 17 parts": (30000, 33, {"slots_override": 2048, "alpha": 0.9, "hash128": 1}),
    "128-bit hash, Vec": (6000, 34, {"hash128": 1, "remap": O.REMAP_VEC}),
}


@pytest.mark.parametrize("name", sorted(STRING_CASES))
def test_string_query_equals_the_big_integer_restatement(name):
    n, seed, params = STRING_CASES[name]
    data, off = W.strings(torch.arange(n), seed=seed)
    d, o = data.numpy(), off.numpy().astype(np.uint64)
    m = O.OracleMPHF.build_bytes(d, o, **params)
    st = R.parse(m.serialize())
    assert st.key_kind == 1 and st.hash128 == bool(params.get("hash128", 0))
    ids = np.concatenate([_sample(n, 1500, seed), n + np.arange(500)])   # ids >= n are other strings
    qd, qo = W.strings(torch.from_numpy(ids), seed=seed)
    qd, qo = qd.numpy(), qo.numpy().astype(np.uint64)
    got = m.query_bytes(qd, qo).tolist()
    for i in range(len(ids)):
        s = qd[qo[i]:qo[i + 1]].tobytes()
        assert O.hash_bytes(s, st.seed) == R.string_hash(s, st.seed)[1]
        assert got[i] == R.query_bytes(st, s), f"{name}: string {ids[i]}"


def test_restatement_reads_hand_made_cacheline_ef_lines():
    """The CacheLineEF decode of the restatement on lines written by hand
    from Sec. 3.4's definition: value v_i puts bit i + (v_i >> 8) - offset
    of the 128-bit field, offset = v_0 >> 8, low byte v_i mod 256."""
    rng = np.random.default_rng(5)
    for trial in range(50):
        vals = np.sort(rng.integers(0, 256 * 80, size=44))
        offset = int(vals[0]) >> 8
        field = 0
        for i, v in enumerate(vals.tolist()):
            field |= 1 << (i + (v >> 8) - offset)
        line = field.to_bytes(16, "little") + offset.to_bytes(4, "little") + bytes(int(v) & 255 for v in vals)
        st = R.Structure(key_kind=0, gamma=3, remap=0, reduce=0, hash128=False, n=10, P=1, S=64, B=1, C=1,
                         seed=0, remap_len=44, pilots=b"\0", remap_payload=line)
        assert [R.remap_entry(st, j) for j in range(44)] == vals.tolist()
        # and the oracle's own decoder agrees on the same bytes
        arr = np.frombuffer(line, dtype=np.uint8).copy()
        assert [O.clef_get(arr, j) for j in range(44)] == vals.tolist()


def test_restatement_gamma3_and_reduce_on_closed_forms():
    """Spot values of the restatement that follow from the definitions alone:
    gamma_3(0) = 0; gamma_3 at x = 1/2 (2^63) with x^2 = 2^62 and x^3 = 2^61
    exactly; and with one bucket, pilot 0 and seed 0 (so hp = 0) the
    power-of-two slot of h is the high half of C h, masked to log2(S) bits."""
    assert R.gamma_value(3, 0) == 0
    half = 1 << 63
    t = (1 << 62) // 2 + (1 << 61) // 2
    assert R.gamma_value(3, half) == t - t // 256 + half // 256
    st = R.Structure(key_kind=0, gamma=1, remap=1, reduce=0, hash128=False, n=1 << 20, P=1, S=1 << 20, B=1,
                     C=R.K1, seed=0, remap_len=0, pilots=b"\0", remap_payload=b"")
    for h in (0, 1, (1 << 64) - 1, 0x0123456789ABCDEF):
        assert R.slot(st, h, h) == ((R.K1 * h) >> 64) & ((1 << 20) - 1)
