"""PtrHash CPU oracle: ctypes wrapper -- TEST INFRASTRUCTURE ONLY.

Only the test-suite, ``__graft_entry__.smoke()`` and the CPU-baseline legs of
``bench.py`` may import this module.  The product library never does, and the
two share no code: they meet only through the serialized byte format, which
each side reads and writes with its own code.

The C source (``ptrhash_oracle.c``) restates the PtrHash paper: Eq. partbucket
and Eq. slot (Sec. 3.1), the greedy + hash-evict construction (Sec. 3.2),
the bucket functions gamma_1 / gamma_3 (Sec. 3.3) and remapping with
CacheLineEF (Sec. 3.4, Eq. clef).  The string hash is the project's own
definition.  Its finishing mixer is pinned to SplitMix64's published outputs.
Its per-word fold and sum are pinned to the same outputs through words whose
fold has a closed form (inputs 0, 1 and 2^63); at other inputs the fold is
checked by properties only.
"""
from __future__ import annotations

import ctypes
import os
import subprocess
import threading

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "ptrhash_oracle.c")
_LIB = os.path.join(_HERE, "libptrhash_oracle.so")
# A prebuilt library to load instead (the mutation tests load planted mistakes this way).
_LIB_OVERRIDE = os.environ.get("PTRHASH_ORACLE_LIB")

OK = 0
ERR_ARG = -1
ERR_OOM = -2
ERR_DUP_KEYS = -3
ERR_BUILD = -4
ERR_FORMAT = -5
ERR_CLEF_SPAN = -6
ERR_OVERFULL = -7

GAMMA_LINEAR = 1
GAMMA_CUBIC = 3
REMAP_CLEF = 0
REMAP_VEC = 1
REDUCE_POW2 = 0
REDUCE_MOD = 1
KEY_U64 = 0
KEY_BYTES = 1
CLEF_PER_LINE = 44


class OracleError(RuntimeError):
    def __init__(self, code: int, what: str):
        super().__init__(f"{what}: oracle error {code}")
        self.code = code


class Layout(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("P", ctypes.c_uint64), ("S", ctypes.c_uint64),
                ("B", ctypes.c_uint64), ("reduce", ctypes.c_int32), ("pad", ctypes.c_int32)]


class Params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("alpha", ctypes.c_double),
                ("gamma", ctypes.c_int32), ("remap", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("C", ctypes.c_uint64),
                ("slots_override", ctypes.c_uint64), ("max_reseeds", ctypes.c_int32),
                ("evict_mult", ctypes.c_uint32), ("threads", ctypes.c_int32),
                ("hash128", ctypes.c_int32)]


_lock = threading.Lock()
_lib = None


def build_library(force: bool = False) -> str:
    """Compile the oracle with the host C compiler (plain C11 + pthreads)."""
    if _LIB_OVERRIDE:
        return _LIB_OVERRIDE
    if force or not os.path.exists(_LIB) or os.path.getmtime(_LIB) < max(
            os.path.getmtime(_SRC), os.path.getmtime(os.path.join(_HERE, "ptrhash_oracle.h"))):
        tmp = _LIB + f".tmp{os.getpid()}"
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-pthread",
                               "-o", tmp, _SRC, "-lm"])
        os.replace(tmp, _LIB)
    return _LIB


def lib():
    global _lib
    with _lock:
        if _lib is None:
            path = build_library()
            L = ctypes.CDLL(path)
            u64, i32, vp = ctypes.c_uint64, ctypes.c_int, ctypes.c_void_p
            L.orc_hi.restype = u64; L.orc_hi.argtypes = [u64, u64]
            L.orc_lo.restype = u64; L.orc_lo.argtypes = [u64, u64]
            L.orc_gamma.restype = u64; L.orc_gamma.argtypes = [i32, u64]
            L.orc_hash_u64.restype = u64; L.orc_hash_u64.argtypes = [u64, u64]
            L.orc_hash_bytes.restype = u64; L.orc_hash_bytes.argtypes = [vp, u64, u64]
            L.orc_hash_bytes128.restype = None
            L.orc_hash_bytes128.argtypes = [vp, u64, u64, ctypes.POINTER(u64), ctypes.POINTER(u64)]
            L.orc_slot_of_hash2.restype = u64; L.orc_slot_of_hash2.argtypes = [vp, u64, u64]
            L.orc_hp.restype = u64; L.orc_hp.argtypes = [u64, u64, u64]
            L.orc_reduce.restype = u64; L.orc_reduce.argtypes = [i32, u64, u64, u64]
            L.orc_part_bucket.restype = None
            L.orc_part_bucket.argtypes = [ctypes.POINTER(Layout), i32, u64,
                                          ctypes.POINTER(u64), ctypes.POINTER(u64)]
            L.orc_layout_for.restype = i32
            L.orc_layout_for.argtypes = [u64, ctypes.c_double, ctypes.c_double, u64,
                                         ctypes.POINTER(Layout)]
            L.orc_default_params.restype = None
            L.orc_default_params.argtypes = [ctypes.POINTER(Params)]
            L.orc_clef_encode.restype = i32; L.orc_clef_encode.argtypes = [vp, u64, vp]
            L.orc_clef_get.restype = u64; L.orc_clef_get.argtypes = [vp, u64]
            L.orc_build_u64.restype = i32
            L.orc_build_u64.argtypes = [vp, u64, ctypes.POINTER(Params), ctypes.POINTER(vp)]
            L.orc_build_bytes.restype = i32
            L.orc_build_bytes.argtypes = [vp, vp, u64, ctypes.POINTER(Params), ctypes.POINTER(vp)]
            L.orc_free.restype = None; L.orc_free.argtypes = [vp]
            L.orc_slot_of_hash.restype = u64; L.orc_slot_of_hash.argtypes = [vp, u64]
            L.orc_query_hash.restype = u64; L.orc_query_hash.argtypes = [vp, u64]
            L.orc_query_u64_many.restype = None
            L.orc_query_u64_many.argtypes = [vp, vp, u64, vp, i32]
            L.orc_query_bytes_many.restype = None
            L.orc_query_bytes_many.argtypes = [vp, vp, vp, u64, vp, i32]
            L.orc_slot_u64_many.restype = None
            L.orc_slot_u64_many.argtypes = [vp, vp, u64, vp]
            L.orc_serialized_size.restype = u64; L.orc_serialized_size.argtypes = [vp]
            L.orc_serialize.restype = i32; L.orc_serialize.argtypes = [vp, vp, u64]
            L.orc_deserialize.restype = i32
            L.orc_deserialize.argtypes = [vp, u64, ctypes.POINTER(vp)]
            L.orc_get_layout.restype = None
            L.orc_get_layout.argtypes = [vp, ctypes.POINTER(Layout)]
            L.orc_pilots.restype = ctypes.POINTER(ctypes.c_uint8); L.orc_pilots.argtypes = [vp]
            L.orc_remap_len.restype = u64; L.orc_remap_len.argtypes = [vp]
            L.orc_remap_values.restype = None; L.orc_remap_values.argtypes = [vp, vp]
            L.orc_seed.restype = u64; L.orc_seed.argtypes = [vp]
            L.orc_remap_kind.restype = i32; L.orc_remap_kind.argtypes = [vp]
            L.orc_gamma_kind.restype = i32; L.orc_gamma_kind.argtypes = [vp]
            L.orc_total_evictions.restype = u64; L.orc_total_evictions.argtypes = []
            _lib = L
        return _lib


def _ptr(a: np.ndarray) -> int:
    return a.ctypes.data


# ---------------------------------------------------------------- primitives
def hi(a: int, b: int) -> int:
    return lib().orc_hi(a, b)


def lo(a: int, b: int) -> int:
    return lib().orc_lo(a, b)


def gamma(kind: int, x: int) -> int:
    return lib().orc_gamma(kind, x)


def hash_bytes(data: bytes, seed: int) -> int:
    buf = np.frombuffer(data, dtype=np.uint8) if data else np.zeros(1, np.uint8)
    return lib().orc_hash_bytes(_ptr(buf), len(data), seed)


def hash_bytes128(data: bytes, seed: int) -> tuple[int, int]:
    """(hi, lo) of the 128-bit string hash; lo == hash_bytes(data, seed)."""
    buf = np.frombuffer(data, dtype=np.uint8) if data else np.zeros(1, np.uint8)
    hi, lo = ctypes.c_uint64(), ctypes.c_uint64()
    lib().orc_hash_bytes128(_ptr(buf), len(data), seed, ctypes.byref(hi), ctypes.byref(lo))
    return hi.value, lo.value


def reduce(kind: int, C: int, x: int, S: int) -> int:
    return lib().orc_reduce(kind, C, x, S)


def layout_for(n: int, lam: float = 3.5, alpha: float = 0.99, slots_override: int = 0) -> Layout:
    L = Layout()
    rc = lib().orc_layout_for(n, lam, alpha, slots_override, ctypes.byref(L))
    if rc != OK:
        raise OracleError(rc, "layout_for")
    return L


def part_bucket(L: Layout, gamma_kind: int, h: int) -> tuple[int, int]:
    p, b = ctypes.c_uint64(), ctypes.c_uint64()
    lib().orc_part_bucket(ctypes.byref(L), gamma_kind, h, ctypes.byref(p), ctypes.byref(b))
    return p.value, b.value


def clef_encode(vals: np.ndarray) -> np.ndarray:
    vals = np.ascontiguousarray(vals, dtype=np.uint64)
    nlines = (len(vals) + CLEF_PER_LINE - 1) // CLEF_PER_LINE
    out = np.zeros(max(nlines, 1) * 64, dtype=np.uint8)
    rc = lib().orc_clef_encode(_ptr(vals), len(vals), _ptr(out))
    if rc != OK:
        raise OracleError(rc, "clef_encode")
    return out[: nlines * 64]


def clef_get(lines: np.ndarray, j: int) -> int:
    return lib().orc_clef_get(_ptr(lines), j)


def default_params(**kw) -> Params:
    p = Params()
    lib().orc_default_params(ctypes.byref(p))
    for k, v in kw.items():
        setattr(p, "lambda_" if k == "lam" else k, v)
    return p


# ----------------------------------------------------------------- structure
class OracleMPHF:
    """A structure held by the oracle (host memory)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def __del__(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            lib().orc_free(h)
            self._h = None

    # -- construction
    @classmethod
    def build_u64(cls, keys: np.ndarray, **params) -> "OracleMPHF":
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        p = default_params(**params)
        out = ctypes.c_void_p()
        rc = lib().orc_build_u64(_ptr(keys), len(keys), ctypes.byref(p), ctypes.byref(out))
        if rc != OK:
            raise OracleError(rc, "build_u64")
        return cls(out.value)

    @classmethod
    def build_bytes(cls, data: np.ndarray, offsets: np.ndarray, **params) -> "OracleMPHF":
        data = np.ascontiguousarray(data, dtype=np.uint8)
        if data.size == 0:
            data = np.zeros(1, np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        p = default_params(**params)
        out = ctypes.c_void_p()
        rc = lib().orc_build_bytes(_ptr(data), _ptr(offsets), len(offsets) - 1,
                                   ctypes.byref(p), ctypes.byref(out))
        if rc != OK:
            raise OracleError(rc, "build_bytes")
        return cls(out.value)

    @classmethod
    def deserialize(cls, blob: bytes) -> "OracleMPHF":
        buf = np.frombuffer(blob, dtype=np.uint8)
        out = ctypes.c_void_p()
        rc = lib().orc_deserialize(_ptr(buf), len(buf), ctypes.byref(out))
        if rc != OK:
            raise OracleError(rc, "deserialize")
        return cls(out.value)

    def serialize(self) -> bytes:
        size = lib().orc_serialized_size(self._h)
        buf = np.zeros(size, dtype=np.uint8)
        rc = lib().orc_serialize(self._h, _ptr(buf), size)
        if rc != OK:
            raise OracleError(rc, "serialize")
        return buf.tobytes()

    # -- description
    @property
    def layout(self) -> Layout:
        L = Layout()
        lib().orc_get_layout(self._h, ctypes.byref(L))
        return L

    @property
    def n(self) -> int:
        return self.layout.n

    @property
    def seed(self) -> int:
        return lib().orc_seed(self._h)

    @property
    def remap_kind(self) -> int:
        return lib().orc_remap_kind(self._h)

    @property
    def gamma_kind(self) -> int:
        return lib().orc_gamma_kind(self._h)

    def pilots(self) -> np.ndarray:
        L = self.layout
        ptr = lib().orc_pilots(self._h)
        return np.ctypeslib.as_array(ptr, shape=(L.P * L.B,)).copy()

    @property
    def wide(self) -> bool:
        """Values pass 32 bits (n > 2^32): results come as uint64, else uint32."""
        return self.layout.n > (1 << 32)

    def _values(self, out: np.ndarray) -> np.ndarray:
        return out if self.wide else out.astype(np.uint32)

    def remap_values(self) -> np.ndarray:
        m = lib().orc_remap_len(self._h)
        out = np.zeros(max(m, 1), dtype=np.uint64)
        lib().orc_remap_values(self._h, _ptr(out))
        return self._values(out[:m])

    # -- queries, one key at a time
    def query_u64(self, keys: np.ndarray, threads: int = 1) -> np.ndarray:
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(max(len(keys), 1), dtype=np.uint64)
        lib().orc_query_u64_many(self._h, _ptr(keys), len(keys), _ptr(out), threads)
        return self._values(out[: len(keys)])

    def query_bytes(self, data: np.ndarray, offsets: np.ndarray, threads: int = 1) -> np.ndarray:
        data = np.ascontiguousarray(data, dtype=np.uint8)
        if data.size == 0:
            data = np.zeros(1, np.uint8)
        offsets = np.ascontiguousarray(offsets, dtype=np.uint64)
        cnt = len(offsets) - 1
        out = np.zeros(max(cnt, 1), dtype=np.uint64)
        lib().orc_query_bytes_many(self._h, _ptr(data), _ptr(offsets), cnt, _ptr(out), threads)
        return self._values(out[:cnt])

    def slots_u64(self, keys: np.ndarray) -> np.ndarray:
        """PHF (non-minimal) values: the slot before remapping."""
        keys = np.ascontiguousarray(keys, dtype=np.uint64)
        out = np.zeros(max(len(keys), 1), dtype=np.uint64)
        lib().orc_slot_u64_many(self._h, _ptr(keys), len(keys), _ptr(out))
        return out[: len(keys)]

    def query_hash(self, h: int) -> int:
        return lib().orc_query_hash(self._h, h)

    def slot_of_hash(self, h: int) -> int:
        return lib().orc_slot_of_hash(self._h, h)


def last_build_evictions() -> int:
    return lib().orc_total_evictions()
