"""Pins of the CPU oracle against what the paper and the mathematics fix.

Each test names the passage it pins.  None of them re-calls the oracle's own
routine to produce an expected value: the expectations are closed forms in
exact integer / rational arithmetic, invariants, brute force on tiny inputs,
or numbers printed in the paper's tables.
"""
from __future__ import annotations

import math
import os
import random
from fractions import Fraction

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W

M64 = (1 << 64) - 1
C_DEFAULT = 0x9E3779B97F4A7C15
GOLDEN = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def golden_rows(name):
    """Whitespace-separated rows of a fixture under tests/golden/ ('#' starts a comment)."""
    with open(os.path.join(GOLDEN, name)) as f:
        return [line.split() for line in f if line.strip() and not line.lstrip().startswith("#")]


SPACE = {(r[0], int(r[1]), float(r[2]), r[3]): float(r[4]) for r in golden_rows("space_bits_per_key.txt")}


def keys_np(n, seed=0):
    return W.as_uint64_numpy(W.u64_keys(n, seed))


# ------------------------------------------------------------------ Sec. 3.1
def test_hi_lo_are_the_128_bit_product_halves():
    """hi(a*b) and lo(a*b): the high / low 64 bits of the exact product (Sec. 3.1)."""
    rng = random.Random(1)
    vals = [0, 1, 2, M64, M64 - 1, 1 << 63, (1 << 63) - 1, C_DEFAULT]
    vals += [rng.getrandbits(64) for _ in range(200)]
    for a in vals:
        b = rng.getrandbits(64)
        assert O.hi(a, b) == (a * b) >> 64
        assert O.lo(a, b) == (a * b) & M64
        assert O.hi(a, b) * (1 << 64) + O.lo(a, b) == a * b


@pytest.mark.parametrize("n", [10_000_000, 1_000_000_000])
def test_part_is_fast_range_with_exact_boundaries(n):
    """part = hi(P*h) = floor(P h / 2^64): part i starts at ceil(i 2^64 / P) (Eq. partbucket)."""
    L = O.layout_for(n)
    P = L.P
    for i in list(range(1, min(P, 50))) + [P - 1]:
        h0 = -((-i << 64) // P)  # ceil(i * 2^64 / P)
        assert O.part_bucket(L, O.GAMMA_CUBIC, h0)[0] == i
        assert O.part_bucket(L, O.GAMMA_CUBIC, h0 - 1)[0] == i - 1
    assert O.part_bucket(L, O.GAMMA_CUBIC, 0)[0] == 0
    assert O.part_bucket(L, O.GAMMA_CUBIC, M64)[0] == P - 1


def test_bucket_of_linear_gamma_has_exact_boundaries():
    """With gamma_1 and one part, bucket = floor(B h / 2^64) (Eq. partbucket, Sec. 3.3)."""
    L = O.layout_for(20_000)  # small n: a single part
    assert L.P == 1
    B = L.B
    for b in list(range(1, min(B, 300))) + [B - 1]:
        x0 = -((-b << 64) // B)
        assert O.part_bucket(L, O.GAMMA_LINEAR, x0) == (0, b)
        assert O.part_bucket(L, O.GAMMA_LINEAR, x0 - 1) == (0, b - 1)


def test_bucket_uses_the_relative_position_inside_the_part():
    """x = lo(P*h)/2^64 is the position of h inside its part (Eq. partbucket):
    the first hash of every part lands in bucket 0 and the last in bucket B-1."""
    L = O.layout_for(50_000_000)
    for i in range(L.P):
        first = -((-i << 64) // L.P)
        last = -((-(i + 1) << 64) // L.P) - 1
        for g in (O.GAMMA_LINEAR, O.GAMMA_CUBIC):
            assert O.part_bucket(L, g, first) == (i, 0)
            assert O.part_bucket(L, g, last) == (i, L.B - 1)


# ------------------------------------------------------------------ Sec. 3.3
def gamma3_exact(x: int) -> Fraction:
    t = Fraction(x, 1 << 64)
    return (Fraction(255, 256) * (t * t + t * t * t) / 2 + t / 256) * (1 << 64)


def test_gamma3_matches_its_closed_form():
    """gamma_3(x) = 255/256 (x^2+x^3)/2 + x/256 on fractions of 2^64 (Sec. 3.3).
    The fixed-point value may only lose the few units of the floors it takes."""
    rng = random.Random(7)
    xs = [0, 1, 255, 256, 1 << 32, 1 << 63, M64, M64 - 1]
    xs += [rng.getrandbits(64) for _ in range(2000)]
    xs += [rng.getrandbits(20) for _ in range(200)]
    for x in xs:
        g = O.gamma(O.GAMMA_CUBIC, x)
        exact = gamma3_exact(x)
        assert 0 <= g <= M64
        assert abs(g - exact) <= 4, (x, g, float(exact))


def test_gamma_shapes():
    """gamma_1 is the identity; gamma_3 is monotone, below x, slope 1/256 at 0 (Sec. 3.3)."""
    rng = random.Random(3)
    xs = sorted(rng.getrandbits(64) for _ in range(5000))
    g = [O.gamma(O.GAMMA_CUBIC, x) for x in xs]
    assert all(a <= b for a, b in zip(g, g[1:]))
    assert all(gi <= x for gi, x in zip(g, xs))
    for x in xs[:100]:
        assert O.gamma(O.GAMMA_LINEAR, x) == x
    for e in (8, 20, 31):  # x < 2^32: hi(x*x) = 0, so only the x/256 term is left
        assert O.gamma(O.GAMMA_CUBIC, 1 << e) == (1 << e) >> 8


def test_reduce_definitions():
    """reduce(x,S) = hi(C x) mod S for S = 2^k, x mod S otherwise (Sec. 3.1)."""
    rng = random.Random(5)
    for _ in range(500):
        x = rng.getrandbits(64)
        k = rng.randrange(1, 33)
        assert O.reduce(O.REDUCE_POW2, C_DEFAULT, x, 1 << k) == ((C_DEFAULT * x) >> 64) % (1 << k)
        S = rng.randrange(3, 1 << 32) | 1
        assert O.reduce(O.REDUCE_MOD, C_DEFAULT, x, S) == x % S


# -------------------------------------------------------- parameter rule, Sec. 3.1
def test_layout_at_1e9_follows_the_rule():
    """alpha S >= 80000 ln(n/80000), S = 2^k, P = ceil(n/(alpha S)), B = ceil(alpha S/lambda)."""
    L = O.layout_for(10**9, 3.5, 0.99)
    kpp = 80000 * math.log(10**9 / 80000)
    assert L.S == 1 << 20 and (L.S // 2) * 0.99 < kpp <= L.S * 0.99
    assert L.P == math.ceil(10**9 / (0.99 * L.S)) == 964
    assert L.B == math.ceil(0.99 * L.S / 3.5) == 296_598
    assert L.reduce == O.REDUCE_POW2


def bits_per_key(L, lam_remap):
    n = L.n
    pilots = 8 * L.P * L.B / n
    R = L.P * L.S - n
    clef = 512 * math.ceil(R / 44) / n
    vec = 32 * R / n
    return pilots, clef, vec


@pytest.mark.parametrize("lam", [3.0, 3.5, 4.0])
def test_space_matches_table_remap(lam):
    """Table remap (n = 1e9): pilots 2.67 / 2.29 / 2.00 bits/key, Vec 0.33, CacheLineEF 0.12.
    The table's remap sizes are those of S = 2^18 (the setting of the bucket-function
    figure); with S = 2^18 every figure is reproduced to the printed digits, and the
    parameter rule's S = 2^20 stays within 0.02 of each."""
    pilots_paper = SPACE[("remap", 10**9, lam, "pilots")]
    clef_paper, vec_paper = SPACE[("remap", 10**9, 3.5, "clef")], SPACE[("remap", 10**9, 3.5, "vec")]
    L18 = O.layout_for(10**9, lam, 0.99, slots_override=1 << 18)
    p, c, v = bits_per_key(L18, lam)
    assert round(p, 2) == pilots_paper
    assert round(c, 2) == clef_paper and round(v, 2) == vec_paper
    L20 = O.layout_for(10**9, lam, 0.99)
    p, c, v = bits_per_key(L20, lam)
    assert abs(p - pilots_paper) < 0.02 and abs(c - clef_paper) < 0.02 and abs(v - vec_paper) < 0.02


@pytest.mark.parametrize("lam,remap", [(3.0, "vec"), (3.5, "clef"), (4.0, "clef")])
def test_space_matches_table_comparison(lam, remap):
    """Table comparison (3e8 strings): Fast 2.99, Default 2.40, Compact 2.12 bits/key."""
    total_paper = SPACE[("comparison", 3 * 10**8, lam, "total")]
    L = O.layout_for(3 * 10**8, lam, 0.99)
    p, c, v = bits_per_key(L, lam)
    total = p + (c if remap == "clef" else v)
    assert round(total, 2) == total_paper


def test_layout_small_n_uses_mod_reduce():
    """Few parts: S need not be a power of two and reduce is x mod S (Sec. 3.1)."""
    for n in [1, 2, 3, 10, 23, 1000, 80_000, 100_000, 300_000]:
        L = O.layout_for(n)
        assert L.P * L.S >= n / 0.99 - 1
        assert L.P * L.S <= 1.05 * n / 0.99 + 18 * L.P  # at most 16 extra spare slots
        assert L.S - -(-n // L.P) >= 16
        if L.reduce == O.REDUCE_MOD:
            assert L.S & (L.S - 1) != 0 and L.S % 2 == 1
    assert O.layout_for(1000).P == 1


@pytest.mark.parametrize("n", [1000, 20_000, 100_000, 300_000])
@pytest.mark.parametrize("t", [1, 8, 20, 32])
def test_x_mod_s_reaches_every_residue_for_keys_with_trailing_zeros(n, t):
    """Sec. 3.1 wants x mod S to depend on every bit of x. Keys k 2^t hash to h = C k 2^t,
    which ends in t zero bits, so for one pilot x = h xor hp keeps hp's low t bits on every
    key. With an even S those keys would reach only S / gcd(S, 2^t) residues; the layout's S
    is odd, so brute force over the keys must find residues well spread over [0, S)."""
    L = O.layout_for(n)
    assert L.reduce == O.REDUCE_MOD
    assert math.gcd(L.S, 1 << t) == 1
    keys = (np.arange(n, dtype=np.uint64) * np.uint64(7919) + np.uint64(1)) << np.uint64(t)   # < 2^64: distinct
    hp = (C_DEFAULT * 3) & M64
    residues = {((C_DEFAULT * int(k)) & M64 ^ hp) % L.S for k in keys.tolist()}
    assert len(residues) >= min(n, L.S) * 0.6


@pytest.mark.parametrize("t", [8, 20])
def test_small_layout_builds_keys_with_trailing_zeros(t):
    """n = 1000 keys k 2^t: with an even S = 1016 they could reach at most 1016 / 8 = 127
    slots and no build could succeed; with the odd S every slot is reachable and these
    builds succeed. (Structured key sets can still defeat the pilot search for other
    reasons, e.g. t = 3 here; such keys should be passed through a bijective mixer first.)"""
    n = 1000
    keys = np.arange(1, n + 1, dtype=np.uint64) << np.uint64(t)
    ref = O.OracleMPHF.build_u64(keys, threads=2, max_reseeds=3)
    assert np.array_equal(np.sort(ref.query_u64(keys)), np.arange(n, dtype=np.uint32))


# ------------------------------------------------------------------ Sec. 3.4
def random_monotone(rng, m, max_gap):
    v = rng.randrange(0, 1 << 32)
    out = []
    for _ in range(m):
        v += rng.randrange(0, max_gap + 1)
        out.append(v)
    return np.array(out, dtype=np.uint64)


def bits_of(line):
    w0 = int.from_bytes(line[0:8].tobytes(), "little")
    w1 = int.from_bytes(line[8:16].tobytes(), "little")
    return w0 | (w1 << 64)


@pytest.mark.parametrize("m", [1, 2, 43, 44, 45, 88, 1000, 4321])
def test_clef_round_trip_and_layout(m):
    """Eq. clef: each value = 2^8 (offset + select(i) - i) + low[i]; 44 values per 64 B."""
    rng = random.Random(m)
    vals = random_monotone(rng, m, 400)
    lines = O.clef_encode(vals)
    assert len(lines) == 64 * math.ceil(m / 44)
    for j in range(m):
        assert O.clef_get(lines, j) == int(vals[j])
    for c in range(len(lines) // 64):
        line = lines[64 * c: 64 * (c + 1)]
        bits = bits_of(line)
        assert bin(bits).count("1") == 44            # one distinct bit per value
        v0 = int(vals[44 * c])
        assert int.from_bytes(line[16:20].tobytes(), "little") == v0 >> 8
        for i in range(44):
            vi = int(vals[min(44 * c + i, m - 1)])
            assert line[20 + i] == vi & 0xFF
            # bit i + high(v_i) - high(v_0) is set (brute-force select)
            assert (bits >> (i + (vi >> 8) - (v0 >> 8))) & 1


def test_clef_span_and_width_limits():
    """Span: bit 43 + (high(v43) - high(v0)) must be < 128; values <= 40 bits (Sec. 3.4)."""
    base = 1 << 20
    ok = np.array([base] * 43 + [base + 84 * 256], dtype=np.uint64)  # last bit = 127
    lines = O.clef_encode(ok)
    assert O.clef_get(lines, 43) == base + 84 * 256
    bad = np.array([base] * 43 + [base + 85 * 256], dtype=np.uint64)  # would need bit 128
    with pytest.raises(O.OracleError) as e:
        O.clef_encode(bad)
    assert e.value.code == O.ERR_CLEF_SPAN
    with pytest.raises(O.OracleError) as e:
        O.clef_encode(np.array([1 << 40], dtype=np.uint64))
    assert e.value.code == O.ERR_ARG
    with pytest.raises(O.OracleError):
        O.clef_encode(np.array([5, 4], dtype=np.uint64))  # not non-decreasing
    assert abs(64 * 8 / 44 - 11.6) < 0.05  # 11.6 bits per value


# ------------------------------------------------- MPHF definition (Sec. 1)
SMALL_NS = [1, 2, 3, 4, 5, 7, 10, 23, 64, 100, 257, 1000, 1999, 2000]


@pytest.mark.parametrize("n", SMALL_NS)
def test_bijection_brute_force_small_n(n):
    """An MPHF maps the n keys bijectively onto [0, n) (Sec. 1, problem statement)."""
    keys = keys_np(n, seed=n)
    m = O.OracleMPHF.build_u64(keys)
    out = m.query_u64(keys)
    assert sorted(out.tolist()) == list(range(n))


# A forced small S gives many parts at small n.  gamma_3's slope of 1/256 at 0
# is tuned for parts of 2^18..2^20 slots, so the forced parts keep >= 1024
# slots, and alpha <= 0.9 keeps every part's key count below S despite the
# binomial spread of part sizes (u64 keys cannot be reseeded into other parts).
@pytest.mark.parametrize("n,S,gamma,remap,alpha", [
    (30000, 2048, O.GAMMA_CUBIC, O.REMAP_CLEF, 0.9),   # 17 parts, power-of-two S
    (20000, 1024, O.GAMMA_LINEAR, O.REMAP_VEC, 0.9),   # Fast-style
    (30000, 3001, O.GAMMA_CUBIC, O.REMAP_CLEF, 0.9),   # x mod S with several parts
    (50000, 4096, O.GAMMA_CUBIC, O.REMAP_VEC, 0.95),
])
def test_bijection_many_parts(n, S, gamma, remap, alpha):
    keys = keys_np(n, seed=11)
    m = O.OracleMPHF.build_u64(keys, slots_override=S, gamma=gamma, remap=remap, alpha=alpha)
    L = m.layout
    assert L.P > 1 and L.S == S
    out = m.query_u64(keys)
    assert np.array_equal(np.sort(out), np.arange(n, dtype=np.uint32))


def test_slots_stay_inside_their_part_and_pilot_xor_seed():
    """slot = part*S + reduce(h xor C (p xor seed), S) (Eq. slot, Eq. hp):
    every slot lies in its part's range, and pilot p under seed s acts as pilot
    p xor s xor s' under seed s' (the xor form of hp)."""
    n = 20000
    keys = keys_np(n, seed=3)
    m0 = O.OracleMPHF.build_u64(keys, slots_override=1024, seed=0, alpha=0.85)
    L = m0.layout
    slots = m0.slots_u64(keys)
    C = C_DEFAULT
    parts = np.array([O.hi(L.P, (C * int(k)) & M64) for k in keys])
    assert np.all(slots // L.S == parts)
    # Rebuild a structure by hand with seed 1 and pilots p xor 1: same slots.
    blob = bytearray(m0.serialize())
    pil = np.frombuffer(bytes(blob[128:128 + L.P * L.B]), dtype=np.uint8)
    blob[72:80] = (1).to_bytes(8, "little")
    blob[128:128 + L.P * L.B] = (pil ^ 1).tobytes()
    m1 = O.OracleMPHF.deserialize(bytes(blob))
    assert np.array_equal(m1.slots_u64(keys), slots)


def test_remap_invariants():
    """Remap (Sec. 3.4): the keys beyond n are sent, in order, to the free slots < n;
    F is non-decreasing; undefined entries repeat their predecessor."""
    n = 20000
    keys = keys_np(n, seed=5)
    for remap in (O.REMAP_CLEF, O.REMAP_VEC):
        m = O.OracleMPHF.build_u64(keys, slots_override=2048, remap=remap, alpha=0.9)
        L = m.layout
        slots = m.slots_u64(keys)
        assert len(np.unique(slots)) == n                 # a perfect hash first
        F = m.remap_values().astype(np.int64)
        assert len(F) == L.P * L.S - n
        assert np.all(np.diff(F) >= 0)
        high = np.sort(slots[slots >= n])
        taken_low = np.zeros(n, dtype=bool)
        taken_low[slots[slots < n]] = True
        free_low = np.flatnonzero(~taken_low)
        assert len(high) == len(free_low)                  # |{q >= n}| = |{free < n}| = R
        assert np.array_equal(F[high - n], free_low)       # F[q_i - n] = L_i
        out = m.query_u64(keys)
        assert np.array_equal(np.sort(out), np.arange(n))


def test_nonmember_queries_are_total_and_in_range():
    n = 3000
    keys = keys_np(n)
    m = O.OracleMPHF.build_u64(keys)
    other = W.as_uint64_numpy(W.nonmember_u64_keys(10000, n))
    out = m.query_u64(other)
    assert out.max() < n


def test_pilots_are_bytes_and_buckets_cover_keys():
    """Pilots are 8-bit (Sec. 3.1); every key's bucket index is in [0, P*B)."""
    n = 10000
    keys = keys_np(n)
    m = O.OracleMPHF.build_u64(keys, slots_override=2048, alpha=0.9)
    L = m.layout
    assert m.pilots().dtype == np.uint8 and len(m.pilots()) == L.P * L.B
    for k in keys[:500]:
        p, b = O.part_bucket(L, O.GAMMA_CUBIC, (C_DEFAULT * int(k)) & M64)
        assert 0 <= p < L.P and 0 <= b < L.B


# ---------------------------------------------------------- failure paths
def test_duplicate_keys_are_rejected():
    keys = keys_np(1000)
    keys[10] = keys[500]
    with pytest.raises(O.OracleError) as e:
        O.OracleMPHF.build_u64(keys)
    assert e.value.code == O.ERR_DUP_KEYS


def test_eviction_cap_fails_cleanly():
    """Construction gives up after evict_mult * S evictions (Sec. 4.1.2); the same
    keys build under the default cap of 10 S, using hash-evict (Sec. 3.2)."""
    keys = keys_np(200_000, seed=4)
    m = O.OracleMPHF.build_u64(keys, max_reseeds=0)
    assert O.last_build_evictions() > 0
    out = m.query_u64(keys)
    assert np.array_equal(np.sort(out), np.arange(len(keys)))
    with pytest.raises(O.OracleError) as e:
        O.OracleMPHF.build_u64(keys, evict_mult=0, max_reseeds=0)
    assert e.value.code == O.ERR_BUILD


def test_bad_arguments():
    with pytest.raises(O.OracleError):
        O.OracleMPHF.build_u64(np.zeros(0, np.uint64))
    with pytest.raises(O.OracleError):
        O.OracleMPHF.build_u64(keys_np(10), C=2)  # C must be odd


def test_serialize_round_trip_and_corruption():
    keys = keys_np(5000)
    m = O.OracleMPHF.build_u64(keys, slots_override=1024, alpha=0.85)
    blob = m.serialize()
    m2 = O.OracleMPHF.deserialize(blob)
    assert np.array_equal(m.query_u64(keys), m2.query_u64(keys))
    bad = bytearray(blob)
    bad[0] = ord("X")
    with pytest.raises(O.OracleError):
        O.OracleMPHF.deserialize(bytes(bad))
    bad = bytearray(blob)
    bad[40] ^= 1  # P changes: P*B no longer matches
    with pytest.raises(O.OracleError):
        O.OracleMPHF.deserialize(bytes(bad))
    with pytest.raises(O.OracleError):
        O.OracleMPHF.deserialize(blob[:-1])


# ---------------------------------------------------------------- strings
def test_empty_string_hash_is_the_splitmix64_mixer_of_the_seed():
    """The hash finishes with the SplitMix64 mixer (tests/golden/splitmix64_seed0.txt). An empty
    string has no words and length 0, so its hash is that mixer applied to the seed; with seed
    k * 0x9E3779B97F4A7C15 it equals the generator's k-th output from state 0. The high half of the
    128-bit hash is the same construction with seed xor K4."""
    k4 = 0x47523634D9D6709B
    for k, want in ((int(r[0]), int(r[1], 16)) for r in golden_rows("splitmix64_seed0.txt")):
        seed = (k * 0x9E3779B97F4A7C15) & M64
        assert O.hash_bytes(b"", seed) == want
        hi, lo = O.hash_bytes128(b"", seed ^ k4)
        assert hi == want


def test_string_hash_words_are_pinned_by_splitmix64():
    """The per-word part of the string hash, pinned through the SplitMix64 outputs
    (tests/golden/splitmix64_seed0.txt).  For word inputs 0, 1 and 2^63 the fold's
    128-bit product x K collapses to shifts: fold(0) = 0, fold(1) = K and, K being
    odd, fold(2^63) = (K >> 1) xor 2^63.  Strings are built whose words, xored with
    their tweaks seed + j K1, are such inputs; the seed is then chosen so that the
    finisher's input acc xor len K2 xor seed is k * 0x9E3779B97F4A7C15, whose mix
    is the generator's k-th output.  A wrong word order, tweak, fold half, word
    combination or length term gives another value.  The high half of the 128-bit
    hash is checked the same way with its seed xor K4 and its fold constant K5."""
    K1, K2 = 0x9E3779B97F4A7C15, 0xC2B2AE3D27D4EB4F
    K3, K4, K5 = 0xA173621FA8385BE3, 0x47523634D9D6709B, 0x2EF8175451B07575
    le = lambda x: (x & M64).to_bytes(8, "little")
    for k, want in ((int(r[0]), int(r[1], 16)) for r in golden_rows("splitmix64_seed0.txt")):
        target = (k * 0x9E3779B97F4A7C15) & M64
        for K, seed_xor in ((K3, 0), (K5, K4)):
            cases = (((0,), 0), ((1,), K), ((1 << 63,), (K >> 1) ^ (1 << 63)),
                     ((1, 1), (2 * K) & M64), ((0, 1, 0), K))
            for inputs, acc in cases:
                n = 8 * len(inputs)
                inner = target ^ acc ^ ((n * K2) & M64)   # the seed inside the word hash
                s = b"".join(le(x ^ (inner + j * K1)) for j, x in enumerate(inputs))
                if seed_xor == 0:
                    assert O.hash_bytes(s, inner) == want, (k, inputs)
                else:
                    hi, lo = O.hash_bytes128(s, inner ^ seed_xor)
                    assert hi == want, (k, inputs)


def test_string_hash_properties():
    """Project string hash: depends on every byte, on the length and on the seed."""
    rng = random.Random(9)
    s = bytes(rng.randrange(32, 127) for _ in range(40))
    h = O.hash_bytes(s, 0)
    for i in range(len(s)):
        t = bytearray(s)
        t[i] ^= 1
        assert O.hash_bytes(bytes(t), 0) != h
    assert O.hash_bytes(s + b"\0", 0) != h
    assert O.hash_bytes(s[:-1], 0) != h
    assert O.hash_bytes(s, 1) != h
    assert O.hash_bytes(b"", 0) != O.hash_bytes(b"\0", 0)


def test_string_hash_is_collision_free_and_uniform_on_random_strings():
    ids = torch.arange(100_000)
    data, off = W.strings(ids, seed=0)
    data, off = data.numpy(), off.numpy()
    hs = np.array([O.hash_bytes(data[off[i]:off[i + 1]].tobytes(), 0) for i in range(len(ids))],
                  dtype=np.uint64)
    assert len(np.unique(hs)) == len(hs)
    top = (hs >> np.uint64(60)).astype(np.int64)   # 16 equal ranges of [2^64]
    counts = np.bincount(top, minlength=16)
    exp = len(hs) / 16
    chi2 = float(((counts - exp) ** 2 / exp).sum())
    assert chi2 < 45  # 15 dof; p ~ 1e-4


@pytest.mark.parametrize("n", [1, 5, 100, 3000])
def test_string_bijection(n):
    ids = torch.arange(n)
    data, off = W.strings(ids, seed=2)
    m = O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64))
    out = m.query_bytes(data.numpy(), off.numpy().astype(np.uint64))
    assert sorted(out.tolist()) == list(range(n))


def test_duplicate_strings_are_rejected():
    ids = torch.tensor([0, 1, 2, 1])
    data, off = W.strings(ids, seed=2)
    with pytest.raises(O.OracleError) as e:
        O.OracleMPHF.build_bytes(data.numpy(), off.numpy().astype(np.uint64), max_reseeds=2)
    assert e.value.code == O.ERR_DUP_KEYS


def test_threads_do_not_change_the_structure():
    keys = keys_np(30000)
    a = O.OracleMPHF.build_u64(keys, slots_override=2048, threads=1, alpha=0.85).serialize()
    b = O.OracleMPHF.build_u64(keys, slots_override=2048, threads=4, alpha=0.85).serialize()
    assert a == b


# ------------------------------------------------------ 128-bit string hash
def test_string_hash128_halves():
    """The low half is the 64-bit hash; the high half is a second hash of
    the same bytes that depends on every byte, the length and the seed."""
    rng = random.Random(12)
    s = bytes(rng.randrange(0, 256) for _ in range(37))
    hi, lo = O.hash_bytes128(s, 5)
    assert lo == O.hash_bytes(s, 5) and hi != lo
    for i in range(len(s)):
        t = bytearray(s)
        t[i] ^= 0x80
        assert O.hash_bytes128(bytes(t), 5)[0] != hi
    assert O.hash_bytes128(s + b"\0", 5)[0] != hi
    assert O.hash_bytes128(s, 6)[0] != hi
    assert O.hash_bytes128(b"", 0)[0] != O.hash_bytes128(b"\0", 0)[0]


def test_string_hash128_high_half_is_uniform():
    ids = torch.arange(50_000)
    data, off = W.strings(ids, seed=4)
    data, off = data.numpy(), off.numpy()
    his = np.array([O.hash_bytes128(data[off[i]:off[i + 1]].tobytes(), 0)[0] for i in range(len(ids))],
                   dtype=np.uint64)
    assert len(np.unique(his)) == len(his)
    counts = np.bincount((his >> np.uint64(60)).astype(np.int64), minlength=16)
    exp = len(his) / 16
    assert float(((counts - exp) ** 2 / exp).sum()) < 45   # 15 dof; p ~ 1e-4


@pytest.mark.parametrize("n,params", [(1, {}), (300, {}), (20_000, {}),
                                      (30_000, {"slots_override": 2048, "alpha": 0.9})])   # 17 parts
def test_string_build_with_128_bit_hash(n, params):
    """Byte keys with the 128-bit hash (forced here; automatic past 2^32
    keys): the high half picks part and bucket, the low half the slot; the
    result is still a bijection, and the flag survives serialization."""
    data, off = W.strings(torch.arange(n), seed=8)
    d, o = data.numpy(), off.numpy().astype(np.uint64)
    m = O.OracleMPHF.build_bytes(d, o, hash128=1, **params)
    got = m.query_bytes(d, o)
    assert sorted(got.tolist()) == list(range(n))
    blob = m.serialize()
    assert int.from_bytes(blob[28:32], "little") == 1
    m2 = O.OracleMPHF.deserialize(blob)
    assert np.array_equal(m2.query_bytes(d, o), got)
    plain = O.OracleMPHF.build_bytes(d, o, **params)
    assert int.from_bytes(plain.serialize()[28:32], "little") == 0


def test_128_bit_hash_places_keys_by_the_high_half():
    """For a key of a 128-bit structure, its slot follows Eq. partbucket on
    the high half and Eq. slot on the low half: the slot read from the
    structure's own pilot matches, and the part is hi(P * high)."""
    n = 30_000
    data, off = W.strings(torch.arange(n), seed=9)
    d, o = data.numpy(), off.numpy().astype(np.uint64)
    m = O.OracleMPHF.build_bytes(d, o, hash128=1, slots_override=2048, alpha=0.9)   # 17 parts
    L = m.layout
    assert L.P > 1
    for i in range(0, n, 97):
        hi, lo = O.hash_bytes128(d[o[i]:o[i + 1]].tobytes(), m.seed)
        s = O.lib().orc_slot_of_hash2(m._h, hi, lo)
        assert s // L.S == O.hi(L.P, hi)
        part, b = O.part_bucket(L, m.gamma_kind, hi)
        pilot = int(m.pilots()[part * L.B + b])
        C = O.default_params().C
        hp = O.lib().orc_hp(C, m.seed, pilot)
        assert s == part * L.S + O.reduce(L.reduce, C, lo ^ hp, L.S)
