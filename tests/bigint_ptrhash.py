"""PtrHash query restated in plain Python integers, from the paper.

Test infrastructure, independent of both the C oracle and the CUDA library:
it parses the serialized structure byte by byte and evaluates one key at a
time with Python's unbounded integers, so every 64-bit wrap-around and every
high half of a 128-bit product is written out explicitly.  A mistake in the
oracle's C arithmetic (a dropped factor, xor taken for addition, a wrong
half of a product) therefore shows up as a disagreement with this module.

Formulas (PtrHash, SEA 2025):
  * h(k) = C k mod 2^64 for u64 keys (Sec. 3.1, "Hash functions").
  * part = floor(P h / 2^64); x = P h mod 2^64, the position inside the part
    as a fraction of 2^64; bucket = part B + floor(B gamma(x) / 2^64)
    (Eq. partbucket).  gamma_1(x) = x; gamma_3 (Sec. 3.3) on 64-bit fixed
    point: x2 = floor(x^2 / 2^64), x3 = floor(x2 x / 2^64),
    t = floor(x2 / 2) + floor(x3 / 2), gamma = t - floor(t / 256) + floor(x / 256)
    (the reading that every division rounds down).
  * hp(p) = C (p xor seed) mod 2^64 (Eq. hp); slot = part S +
    reduce(h xor hp(p), S) with reduce(y, S) = floor(C y / 2^64) mod S for a
    power-of-two S and y mod S otherwise (Eq. slot, "The reduce function").
  * A slot s >= n returns F[s - n] (Sec. 3.4, "Remapping"); CacheLineEF
    line j // 44 stores v_i = 256 (offset + select(i) - i) + low[i], where
    select(i) is the position of the i-th set bit of the line's 128-bit
    field (Sec. 3.4, Eq. clef and "Lookup").
  * String keys: the project's own hash (the paper uses GxHash and does not
    define it): 8-byte little-endian words w_j zero-padded past the length,
    acc = sum_j fold(w_j xor (seed + j K1)) mod 2^64 with fold(y) = the high
    half xor the low half of y K3, h = splitmix64_finalizer(acc xor len K2
    xor seed).  The 128-bit variant's high half uses seed xor K4 and K5, picks
    the part and bucket; the low half is the 64-bit hash and picks the slot.
"""
from __future__ import annotations

from dataclasses import dataclass

M = 1 << 64
K1 = 0x9E3779B97F4A7C15
K2 = 0xC2B2AE3D27D4EB4F
K3 = 0xA173621FA8385BE3
K4 = 0x47523634D9D6709B
K5 = 0x2EF8175451B07575


def u32(b: bytes, off: int) -> int:
    return int.from_bytes(b[off:off + 4], "little")


def u64(b: bytes, off: int) -> int:
    return int.from_bytes(b[off:off + 8], "little")


@dataclass
class Structure:
    key_kind: int
    gamma: int
    remap: int
    reduce: int
    hash128: bool
    n: int
    P: int
    S: int
    B: int
    C: int
    seed: int
    remap_len: int
    pilots: bytes
    remap_payload: bytes


def parse(blob: bytes) -> Structure:
    """The 128-byte little-endian header, the P*B pilot bytes padded to a
    multiple of 64, then the remap payload."""
    assert blob[:8] == b"PTRHASH1" and u32(blob, 8) == 1
    P, B = u64(blob, 40), u64(blob, 56)
    pilot_bytes = u64(blob, 112)
    assert pilot_bytes == P * B
    start = 128 + (pilot_bytes + 63) // 64 * 64
    remap_bytes = u64(blob, 88)
    return Structure(key_kind=u32(blob, 12), gamma=u32(blob, 16), remap=u32(blob, 20), reduce=u32(blob, 24),
                     hash128=bool(u32(blob, 28) & 1), n=u64(blob, 32), P=P, S=u64(blob, 48), B=B,
                     C=u64(blob, 64), seed=u64(blob, 72), remap_len=u64(blob, 80),
                     pilots=blob[128:128 + pilot_bytes], remap_payload=blob[start:start + remap_bytes])


def gamma_value(kind: int, x: int) -> int:
    if kind == 1:
        return x
    x2 = (x * x) // M
    x3 = (x2 * x) // M
    t = x2 // 2 + x3 // 2
    return t - t // 256 + x // 256


def bucket(st: Structure, hb: int) -> tuple[int, int]:
    """(part, global bucket index) of the hash hb (Eq. partbucket)."""
    part = (st.P * hb) // M
    x = (st.P * hb) % M
    return part, part * st.B + (st.B * gamma_value(st.gamma, x)) // M


def slot(st: Structure, hb: int, hs: int) -> int:
    """The non-minimal slot (Eq. slot); hb = hs except for 128-bit string hashes."""
    part, b = bucket(st, hb)
    pilot = st.pilots[b]
    hp = (st.C * (pilot ^ st.seed)) % M
    y = hs ^ hp
    if st.reduce == 0:
        r = ((st.C * y) // M) % st.S
    else:
        r = y % st.S
    return part * st.S + r


def select(field: int, i: int) -> int:
    """Position of the i-th (0-based) set bit of a 128-bit integer."""
    seen = 0
    for pos in range(128):
        if (field >> pos) & 1:
            if seen == i:
                return pos
            seen += 1
    raise ValueError("fewer set bits than asked for")


def remap_entry(st: Structure, j: int) -> int:
    if st.remap == 1:   # plain array: u32 entries, u64 once n > 2^32
        w = 8 if st.n > (1 << 32) else 4
        return int.from_bytes(st.remap_payload[w * j:w * j + w], "little")
    line = st.remap_payload[64 * (j // 44):64 * (j // 44) + 64]
    i = j % 44
    field = int.from_bytes(line[0:16], "little")
    offset = u32(line, 16)
    return 256 * (offset + select(field, i) - i) + line[20 + i]


def value_of_hash(st: Structure, hb: int, hs: int) -> int:
    s = slot(st, hb, hs)
    return s if s < st.n else remap_entry(st, s - st.n)


def query_u64(st: Structure, key: int) -> int:
    h = (st.C * key) % M
    return value_of_hash(st, h, h)


def _splitmix_finalizer(z: int) -> int:
    z ^= z >> 30
    z = (z * 0xBF58476D1CE4E5B9) % M
    z ^= z >> 27
    z = (z * 0x94D049BB133111EB) % M
    z ^= z >> 31
    return z


def _hash_words(s: bytes, seed: int, k_fold: int) -> int:
    acc = 0
    for j in range((len(s) + 7) // 8):
        w = int.from_bytes(s[8 * j:8 * j + 8].ljust(8, b"\0"), "little")
        y = w ^ ((seed + j * K1) % M)
        prod = y * k_fold
        acc = (acc + ((prod >> 64) ^ (prod % M))) % M
    return _splitmix_finalizer(acc ^ ((len(s) * K2) % M) ^ seed)


def string_hash(s: bytes, seed: int) -> tuple[int, int]:
    """(high, low) of the 128-bit string hash; low is the 64-bit hash."""
    return _hash_words(s, seed ^ K4, K5), _hash_words(s, seed, K3)


def query_bytes(st: Structure, s: bytes) -> int:
    hi, lo = string_hash(s, st.seed)
    return value_of_hash(st, hi if st.hash128 else lo, lo)
