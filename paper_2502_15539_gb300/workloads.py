"""Seeded synthetic workloads shared by the tests, the smoke check and the bench.

This module holds no PtrHash arithmetic.  Every value is a counter-based
function of (seed, index) built from the Murmur3 64-bit finalizer ``fmix64``
(Appleby, MurmurHash3), a bijection on 64-bit integers, evaluated with torch
integer ops so the same call gives the same values on the CPU and on a GPU.

Workload recipes (all seeded):
  * distinct u64 keys:  k_i = fmix64(i xor s_key), i < n  (distinct because
    fmix64 is a bijection; uniform-looking over [0, 2^64)).
  * non-member u64 keys: fmix64(j xor s_key) for j >= n (distinct from every
    member for the same reason).
  * query order: the permutation that sorts fmix64(i xor s_perm).
  * strings: string i has length lo + (fmix64(i xor s_len) >> 8) mod (hi-lo+1)
    and byte t in [0, len) equal to 0x20 + (fmix64((i << 6 | t) xor s_byte) >> 8)
    mod 95 (printable ASCII); packed back to back with u64 offsets.
"""
from __future__ import annotations

import torch

_M64 = (1 << 64) - 1


def _i64(c: int) -> int:
    """A u64 constant as the int64 with the same bit pattern."""
    c &= _M64
    return c - (1 << 64) if c >= (1 << 63) else c


def _lsr(x: torch.Tensor, s: int) -> torch.Tensor:
    """Logical right shift of the u64 bit pattern held in an int64 tensor."""
    return (x >> s) & ((1 << (64 - s)) - 1)


_F1 = _i64(0xFF51AFD7ED558CCD)
_F2 = _i64(0xC4CEB9FE1A85EC53)


def fmix64(x: torch.Tensor) -> torch.Tensor:
    """Murmur3 fmix64 on int64 tensors (two's-complement wrap-around)."""
    x = x ^ _lsr(x, 33)
    x = x * _F1
    x = x ^ _lsr(x, 33)
    x = x * _F2
    x = x ^ _lsr(x, 33)
    return x


def fmix64_int(v: int) -> int:
    """The same finalizer on a Python int (used to derive per-stream salts)."""
    v &= _M64
    v ^= v >> 33
    v = (v * 0xFF51AFD7ED558CCD) & _M64
    v ^= v >> 33
    v = (v * 0xC4CEB9FE1A85EC53) & _M64
    v ^= v >> 33
    return v


def _salt(seed: int, stream: int) -> int:
    return _i64(fmix64_int((seed * 0x9E3779B97F4A7C15 + stream * 0xD1B54A32D192ED03 + 1) & _M64))


_STREAM_KEY, _STREAM_PERM, _STREAM_LEN, _STREAM_BYTE, _STREAM_MISC = 1, 2, 3, 4, 5


def as_uint64_numpy(t: torch.Tensor):
    """Host numpy uint64 view of an int64 tensor's bit patterns."""
    return t.detach().cpu().contiguous().numpy().view("uint64")


def u64_keys(n: int, seed: int = 0, device="cpu", start: int = 0) -> torch.Tensor:
    """Keys start..start+n-1 of the distinct-key stream (int64 bit patterns)."""
    i = torch.arange(start, start + n, dtype=torch.int64, device=device)
    return fmix64(i ^ _salt(seed, _STREAM_KEY))


def u64_keys_at(idx: torch.Tensor, seed: int = 0) -> torch.Tensor:
    """Keys of the given stream indexes (u64_keys(n)[idx] without building it)."""
    return fmix64(idx ^ _salt(seed, _STREAM_KEY))


def nonmember_u64_keys(m: int, n: int, seed: int = 0, device="cpu", start: int = 0) -> torch.Tensor:
    """m keys guaranteed absent from ``u64_keys(n, seed)``."""
    return u64_keys(m, seed, device, start=n + start)


def permutation(n: int, seed: int = 1, device="cpu") -> torch.Tensor:
    """A seeded random permutation of [0, n), identical on every device."""
    i = torch.arange(n, dtype=torch.int64, device=device)
    return torch.argsort(fmix64(i ^ _salt(seed, _STREAM_PERM)))


def uniform_index(m: int, bound: int, seed: int, device="cpu", start: int = 0) -> torch.Tensor:
    """m indexes in [0, bound), counter-based."""
    i = torch.arange(start, start + m, dtype=torch.int64, device=device)
    return _lsr(fmix64(i ^ _salt(seed, _STREAM_MISC)), 8) % bound


def string_lengths(ids: torch.Tensor, seed: int = 0, lo: int = 16, hi: int = 64) -> torch.Tensor:
    return lo + _lsr(fmix64(ids ^ _salt(seed, _STREAM_LEN)), 8) % (hi - lo + 1)


def strings(ids: torch.Tensor, seed: int = 0, lo: int = 16, hi: int = 64,
            chunk_strings: int = 1 << 22):
    """Pack the strings with the given ids (any order) back to back.

    Returns ``(bytes uint8[total], offsets int64[len(ids)+1])`` on ids' device.
    String i is the same wherever it appears, so a permuted ``ids`` gives the
    re-packed query buffer of the same key set.
    """
    if hi > 64:
        raise ValueError("string length above 64 is not supported by this generator")
    dev = ids.device
    lengths = string_lengths(ids, seed, lo, hi)
    offsets = torch.zeros(len(ids) + 1, dtype=torch.int64, device=dev)
    torch.cumsum(lengths, 0, out=offsets[1:])
    total = int(offsets[-1].item())
    out = torch.empty(total, dtype=torch.uint8, device=dev)
    salt = _salt(seed, _STREAM_BYTE)
    for a in range(0, len(ids), chunk_strings):
        b = min(len(ids), a + chunk_strings)
        ln = lengths[a:b]
        base = offsets[a:b]
        owner = torch.repeat_interleave(torch.arange(a, b, device=dev), ln)
        pos = torch.arange(int(offsets[a].item()), int(offsets[b].item()), device=dev)
        t = pos - offsets[owner]
        code = fmix64(((ids[owner] << 6) | t) ^ salt)
        out[int(offsets[a].item()):int(offsets[b].item())] = (0x20 + _lsr(code, 8) % 95).to(torch.uint8)
        del ln, base, owner, pos, t, code
    return out, offsets


def log_uniform_int(m: int, lo: float, hi: float, seed: int, device="cpu") -> torch.Tensor:
    """m integers floor(10^U(log10 lo, log10 hi)), counter-based."""
    import math
    u = uniform_index(m, 1 << 53, seed, device).to(torch.float64) / float(1 << 53)
    return torch.floor(10.0 ** (math.log10(lo) + u * (math.log10(hi) - math.log10(lo)))).to(torch.int64)
