"""Thin ctypes binding of libmphf.so (argument marshalling only).

Every function here forwards to the C entry point of the same name declared
in ``include/mphf.h``; all computation happens in the library's CUDA kernels.
Tensors are torch tensors on the current CUDA device (or pinned host tensors
for ``mphf_query_u64_host``); streams default to torch's current stream.
If the library is missing this module raises instead of falling back.
"""
from __future__ import annotations

import ctypes
import os
import threading

import torch

_HERE = os.path.dirname(os.path.abspath(__file__))
LIB_PATH = os.path.join(_HERE, "libmphf.so")

MPHF_OK = 0
MPHF_ERR_ARG = -1
MPHF_ERR_OOM = -2
MPHF_ERR_DUP_KEYS = -3
MPHF_ERR_BUILD_FAILED = -4
MPHF_ERR_FORMAT = -5
MPHF_ERR_CUDA = -6
MPHF_ERR_TIMEOUT = -7
MPHF_ERR_OVERFULL = -8
MPHF_ERR_CAPACITY = -9

MPHF_KEY_U64 = 0
MPHF_KEY_BYTES = 1
MPHF_GAMMA_LINEAR = 1
MPHF_GAMMA_CUBIC = 3
MPHF_REMAP_CLEF = 0
MPHF_REMAP_VEC = 1


class MphfError(RuntimeError):
    def __init__(self, code: int, what: str, detail: str):
        super().__init__(f"{what} failed: {code} ({detail})")
        self.code = code


class mphf_params(ctypes.Structure):
    _fields_ = [("lambda_", ctypes.c_double), ("alpha", ctypes.c_double),
                ("gamma", ctypes.c_int32), ("remap", ctypes.c_int32),
                ("seed", ctypes.c_uint64), ("C", ctypes.c_uint64),
                ("slots_override", ctypes.c_uint64), ("max_reseeds", ctypes.c_int32),
                ("evict_mult", ctypes.c_uint32), ("shard_keys", ctypes.c_uint64),
                ("hash128", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mphf_info_t(ctypes.Structure):
    _fields_ = [("n", ctypes.c_uint64), ("P", ctypes.c_uint64), ("S", ctypes.c_uint64),
                ("B", ctypes.c_uint64), ("C", ctypes.c_uint64), ("seed", ctypes.c_uint64),
                ("gamma", ctypes.c_int32), ("remap", ctypes.c_int32), ("reduce", ctypes.c_int32),
                ("key_kind", ctypes.c_int32), ("remap_len", ctypes.c_uint64),
                ("pilot_bytes", ctypes.c_uint64), ("remap_bytes", ctypes.c_uint64),
                ("bits_per_key", ctypes.c_double), ("evictions", ctypes.c_uint64),
                ("build_ms", ctypes.c_double), ("build_hash_sort_ms", ctypes.c_double),
                ("build_search_ms", ctypes.c_double), ("build_remap_ms", ctypes.c_double)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class mphf_view_t(ctypes.Structure):
    _fields_ = [("pilots", ctypes.c_void_p), ("remap", ctypes.c_void_p), ("n", ctypes.c_uint64),
                ("P", ctypes.c_uint64), ("S", ctypes.c_uint64), ("B", ctypes.c_uint64), ("C", ctypes.c_uint64),
                ("seed", ctypes.c_uint64), ("barrett", ctypes.c_uint64), ("s_mask", ctypes.c_uint64),
                ("gamma", ctypes.c_int32), ("reduce", ctypes.c_int32), ("remap_kind", ctypes.c_int32),
                ("key_kind", ctypes.c_int32), ("hash128", ctypes.c_int32), ("reserved", ctypes.c_int32)]


class mphf_request(ctypes.Structure):
    _fields_ = [("m", ctypes.c_void_p), ("keys_dev", ctypes.c_void_p), ("offsets_dev", ctypes.c_void_p),
                ("count", ctypes.c_uint64), ("out_dev", ctypes.c_void_p)]


class mphf_batch_config(ctypes.Structure):
    _fields_ = [("keys_per_thread", ctypes.c_int32), ("threads", ctypes.c_int32),
                ("blocks_per_sm", ctypes.c_int32), ("use_graph", ctypes.c_int32)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


class mphf_server_config(ctypes.Structure):
    _fields_ = [("hbm_budget_bytes", ctypes.c_uint64), ("max_batch_requests", ctypes.c_uint32),
                ("max_batch_keys", ctypes.c_uint64), ("slots", ctypes.c_int32)]


class mphf_server_req(ctypes.Structure):
    _fields_ = [("structure", ctypes.c_uint32), ("keys_dev", ctypes.c_void_p), ("offsets_dev", ctypes.c_void_p),
                ("count", ctypes.c_uint64), ("out_dev", ctypes.c_void_p)]


class mphf_server_stats_t(ctypes.Structure):
    _fields_ = [("p50_us", ctypes.c_double), ("p99_us", ctypes.c_double), ("max_us", ctypes.c_double),
                ("mean_us", ctypes.c_double), ("queries_per_s", ctypes.c_double), ("requests", ctypes.c_uint64),
                ("queries", ctypes.c_uint64), ("batches", ctypes.c_uint64),
                ("mean_requests_per_batch", ctypes.c_double), ("admissions", ctypes.c_uint64),
                ("evictions", ctypes.c_uint64), ("resident_bytes", ctypes.c_uint64)]

    def as_dict(self) -> dict:
        return {k: getattr(self, k) for k, _ in self._fields_}


# Exported symbols of include/mphf.h with their ctypes signatures.
_vp, _u64, _i32, _sz = ctypes.c_void_p, ctypes.c_uint64, ctypes.c_int, ctypes.c_size_t
SIGNATURES = {
    "mphf_default_params": (_i32, [ctypes.POINTER(mphf_params)]),
    "mphf_build": (_i32, [ctypes.POINTER(mphf_params), _i32, _vp, _vp, _u64, _vp, ctypes.POINTER(_vp)]),
    "mphf_query_u64": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "mphf_query_bytes": (_i32, [_vp, _vp, _vp, _u64, _vp, _vp]),
    "mphf_query_u64_phf": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "mphf_query_u64_windowed": (_i32, [_vp, _vp, _u64, _vp, _u64, _u64, _vp]),
    "mphf_query_u64_host": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "mphf_serialize": (_i32, [_vp, _vp, _sz, ctypes.POINTER(_sz)]),
    "mphf_deserialize": (_i32, [_vp, _sz, ctypes.POINTER(_vp)]),
    "mphf_info": (_i32, [_vp, ctypes.POINTER(mphf_info_t)]),
    "mphf_free": (None, [_vp]),
    "mphf_strerror": (ctypes.c_char_p, [_i32]),
    "mphf_last_error": (ctypes.c_char_p, []),
    "mphf_layout": (_i32, [ctypes.POINTER(mphf_params), _u64, ctypes.POINTER(mphf_info_t)]),
    "mphf_gather_probe": (_i32, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "mphf_gather_probe_at": (_i32, [_vp, _u64, _vp, _u64, _vp, _vp]),
    "mphf_bucket_u64": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "mphf_launch_count": (_u64, []),
    "mphf_set_l2_fetch_granularity": (_i32, [_i32, ctypes.POINTER(ctypes.c_int)]),
    "mphf_lookup_u64": (_i32, [_vp, _vp, _u64, _vp, ctypes.c_uint32, _vp, _vp]),
    "mphf_build_u64_noalloc": (_i32, [ctypes.POINTER(mphf_params), _vp, _u64, _vp, _sz, ctypes.POINTER(_sz),
                                      _vp]),
    "mphf_batch_create": (_i32, [ctypes.c_uint32, ctypes.POINTER(_vp)]),
    "mphf_batch_run": (_i32, [_vp, ctypes.POINTER(mphf_request), ctypes.c_uint32, _vp]),
    "mphf_batch_set_config": (_i32, [_vp, ctypes.POINTER(mphf_batch_config)]),
    "mphf_batch_get_config": (_i32, [_vp, ctypes.POINTER(mphf_batch_config)]),
    "mphf_batch_autotune": (_i32, [_vp, ctypes.POINTER(mphf_request), ctypes.c_uint32, _vp, ctypes.c_char_p,
                                   ctypes.POINTER(mphf_batch_config)]),
    "mphf_batch_free": (None, [_vp]),
    "mphf_server_default_config": (_i32, [ctypes.POINTER(mphf_server_config)]),
    "mphf_server_create": (_i32, [ctypes.POINTER(mphf_server_config), ctypes.POINTER(_vp)]),
    "mphf_server_add": (_i32, [_vp, _vp, _sz, ctypes.POINTER(ctypes.c_uint32)]),
    "mphf_server_remove": (_i32, [_vp, ctypes.c_uint32]),
    "mphf_server_submit": (_i32, [_vp, ctypes.POINTER(mphf_server_req), ctypes.POINTER(_u64)]),
    "mphf_server_replay": (_i32, [_vp, ctypes.POINTER(mphf_server_req), ctypes.POINTER(ctypes.c_double),
                                  ctypes.c_uint32, ctypes.POINTER(_u64)]),
    "mphf_server_wait": (_i32, [_vp, _u64, _u64, ctypes.POINTER(ctypes.c_int)]),
    "mphf_server_drain": (_i32, [_vp, _u64]),
    "mphf_server_stats": (_i32, [_vp, ctypes.c_int, ctypes.POINTER(mphf_server_stats_t)]),
    "mphf_server_free": (None, [_vp]),
    "mphf_device_view": (_i32, [_vp, ctypes.POINTER(mphf_view_t)]),
    "mphf_query_u64_wide": (_i32, [_vp, _vp, _u64, _vp, _vp]),
    "mphf_query_bytes_wide": (_i32, [_vp, _vp, _vp, _u64, _vp, _vp]),
}

_lock = threading.Lock()
_lib = None


def load(path: str = LIB_PATH) -> ctypes.CDLL:
    """Loads libmphf.so; raises if it has not been built (no fallback)."""
    global _lib
    with _lock:
        if _lib is None:
            if not os.path.exists(path):
                raise RuntimeError(f"{path} is missing: build it with paper_2502_15539_gb300.build_ext.build()")
            lib = ctypes.CDLL(path)
            for name, (res, args) in SIGNATURES.items():
                fn = getattr(lib, name)
                fn.restype = res
                fn.argtypes = args
            _lib = lib
        return _lib


def _check(rc: int, what: str):
    if rc != MPHF_OK:
        lib = load()
        raise MphfError(rc, what, f"{lib.mphf_strerror(rc).decode()}: {lib.mphf_last_error().decode()}")


def _stream(stream) -> int:
    if stream is None:
        return torch.cuda.current_stream().cuda_stream
    return stream.cuda_stream if hasattr(stream, "cuda_stream") else int(stream)


def _dev_ptr(t: torch.Tensor, dtype, what: str) -> int:
    if not t.is_cuda or not t.is_contiguous() or t.dtype != dtype:
        raise ValueError(f"{what}: contiguous {dtype} CUDA tensor required")
    return t.data_ptr()


def _u64_dtype_ok(t: torch.Tensor) -> bool:
    return t.dtype in (torch.int64, getattr(torch, "uint64", torch.int64))


def mphf_default_params(**overrides) -> mphf_params:
    p = mphf_params()
    _check(load().mphf_default_params(ctypes.byref(p)), "mphf_default_params")
    for k, v in overrides.items():
        setattr(p, "lambda_" if k in ("lam", "lambda") else k, v)
    return p


def mphf_layout(n: int, params: mphf_params | None = None) -> dict:
    params = params or mphf_default_params()
    info = mphf_info_t()
    _check(load().mphf_layout(ctypes.byref(params), n, ctypes.byref(info)), "mphf_layout")
    return info.as_dict()


class MPHF:
    """Owns one device-resident structure (mphf_t*)."""

    def __init__(self, handle: int):
        self._h = ctypes.c_void_p(handle)

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mphf_free(h)
            self._h = None

    @property
    def handle(self) -> ctypes.c_void_p:
        return self._h

    def info(self) -> dict:
        return mphf_info(self)

    def serialize(self) -> bytes:
        return mphf_serialize(self)


def mphf_build(keys: torch.Tensor, params: mphf_params | None = None, offsets: torch.Tensor | None = None,
               stream=None) -> MPHF:
    """u64 keys: int64 CUDA tensor; byte keys: uint8 tensor + int64 offsets (n+1)."""
    params = params or mphf_default_params()
    out = ctypes.c_void_p()
    if offsets is None:
        if not _u64_dtype_ok(keys):
            raise ValueError("u64 keys must be an int64 tensor")
        kind, kp, op, n = MPHF_KEY_U64, _dev_ptr(keys, keys.dtype, "keys"), None, keys.numel()
    else:
        kind, kp = MPHF_KEY_BYTES, _dev_ptr(keys, torch.uint8, "bytes")
        op, n = _dev_ptr(offsets, torch.int64, "offsets"), offsets.numel() - 1
    _check(load().mphf_build(ctypes.byref(params), kind, kp, op, n, _stream(stream), ctypes.byref(out)),
           "mphf_build")
    return MPHF(out.value)


def mphf_query_u64_wide(m: MPHF, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """64-bit results (int64 tensor holding the u64 values); any structure."""
    if out is None:
        out = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
    if not _u64_dtype_ok(keys):
        raise ValueError("keys must be int64")
    _check(load().mphf_query_u64_wide(m.handle, _dev_ptr(keys, keys.dtype, "keys"), keys.numel(),
                                      _dev_ptr(out, torch.int64, "out"), _stream(stream)), "mphf_query_u64_wide")
    return out


def mphf_query_bytes_wide(m: MPHF, data: torch.Tensor, offsets: torch.Tensor, out: torch.Tensor | None = None,
                          stream=None) -> torch.Tensor:
    count = offsets.numel() - 1
    if out is None:
        out = torch.empty(count, dtype=torch.int64, device=data.device)
    _check(load().mphf_query_bytes_wide(m.handle, _dev_ptr(data, torch.uint8, "bytes"),
                                        _dev_ptr(offsets, torch.int64, "offsets"), count,
                                        _dev_ptr(out, torch.int64, "out"), _stream(stream)), "mphf_query_bytes_wide")
    return out


def mphf_query_u64(m: MPHF, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    kp = _dev_ptr(keys, keys.dtype, "keys") if _u64_dtype_ok(keys) else None
    if kp is None:
        raise ValueError("keys must be int64")
    _check(load().mphf_query_u64(m.handle, kp, keys.numel(), _dev_ptr(out, torch.int32, "out"), _stream(stream)),
           "mphf_query_u64")
    return out


def mphf_query_u64_windowed(m: MPHF, keys: torch.Tensor, out: torch.Tensor | None = None, window_bytes: int = 0,
                            chunk_keys: int = 0, stream=None) -> torch.Tensor:
    """The windowed evaluation (0: the defaults); the same values as mphf_query_u64."""
    if out is None:
        out = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    _check(load().mphf_query_u64_windowed(m.handle, _dev_ptr(keys, torch.int64, "keys"), keys.numel(),
                                          _dev_ptr(out, torch.int32, "out"), window_bytes, chunk_keys,
                                          _stream(stream)), "mphf_query_u64_windowed")
    return out


def mphf_query_u64_phf(m: MPHF, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    if out is None:
        out = torch.empty(keys.numel(), dtype=torch.int32, device=keys.device)
    _check(load().mphf_query_u64_phf(m.handle, _dev_ptr(keys, torch.int64, "keys"), keys.numel(),
                                     _dev_ptr(out, torch.int32, "out"), _stream(stream)), "mphf_query_u64_phf")
    return out


def mphf_query_bytes(m: MPHF, data: torch.Tensor, offsets: torch.Tensor, out: torch.Tensor | None = None,
                     stream=None) -> torch.Tensor:
    cnt = offsets.numel() - 1
    if out is None:
        out = torch.empty(cnt, dtype=torch.int32, device=offsets.device)
    _check(load().mphf_query_bytes(m.handle, _dev_ptr(data, torch.uint8, "bytes"),
                                   _dev_ptr(offsets, torch.int64, "offsets"), cnt,
                                   _dev_ptr(out, torch.int32, "out"), _stream(stream)), "mphf_query_bytes")
    return out


def mphf_query_u64_host(m: MPHF, keys_host: torch.Tensor, out_host: torch.Tensor | None = None,
                        stream=None) -> torch.Tensor:
    """keys_host / out_host: CPU tensors (pinned for overlapped copies)."""
    if keys_host.is_cuda or keys_host.dtype != torch.int64 or not keys_host.is_contiguous():
        raise ValueError("keys_host: contiguous int64 CPU tensor required")
    if out_host is None:
        out_host = torch.empty(keys_host.numel(), dtype=torch.int32, pin_memory=keys_host.is_pinned())
    _check(load().mphf_query_u64_host(m.handle, keys_host.data_ptr(), keys_host.numel(), out_host.data_ptr(),
                                      _stream(stream)), "mphf_query_u64_host")
    return out_host


def mphf_serialize(m: MPHF) -> bytes:
    lib = load()
    need = ctypes.c_size_t()
    _check(lib.mphf_serialize(m.handle, None, 0, ctypes.byref(need)), "mphf_serialize")
    buf = ctypes.create_string_buffer(need.value)
    _check(lib.mphf_serialize(m.handle, buf, need.value, ctypes.byref(need)), "mphf_serialize")
    return buf.raw


def mphf_deserialize(blob: bytes) -> MPHF:
    out = ctypes.c_void_p()
    _check(load().mphf_deserialize(blob, len(blob), ctypes.byref(out)), "mphf_deserialize")
    return MPHF(out.value)


def mphf_info(m: MPHF) -> dict:
    info = mphf_info_t()
    _check(load().mphf_info(m.handle, ctypes.byref(info)), "mphf_info")
    return info.as_dict()


def mphf_gather_probe(keys: torch.Tensor, table: torch.Tensor, out: torch.Tensor, stream=None) -> torch.Tensor:
    _check(load().mphf_gather_probe(_dev_ptr(keys, torch.int64, "keys"), keys.numel(),
                                    _dev_ptr(table, torch.uint8, "table"), table.numel(),
                                    _dev_ptr(out, torch.int32, "out"), _stream(stream)), "mphf_gather_probe")
    return out


def mphf_gather_probe_at(idx: torch.Tensor, table_ptr: int, table_bytes: int, out: torch.Tensor,
                         stream=None) -> torch.Tensor:
    """out[i] = table[idx[i]]; table_ptr is a device address (for example the
    pilots of mphf_device_view) holding table_bytes bytes."""
    _check(load().mphf_gather_probe_at(_dev_ptr(idx, torch.int64, "idx"), idx.numel(), table_ptr, table_bytes,
                                       _dev_ptr(out, torch.int32, "out"), _stream(stream)), "mphf_gather_probe_at")
    return out


def mphf_bucket_u64(m: MPHF, keys: torch.Tensor, out: torch.Tensor | None = None, stream=None) -> torch.Tensor:
    """Index into the pilot array of each key's bucket (int64 tensor)."""
    if out is None:
        out = torch.empty(keys.numel(), dtype=torch.int64, device=keys.device)
    _check(load().mphf_bucket_u64(m.handle, _dev_ptr(keys, torch.int64, "keys"), keys.numel(),
                                  _dev_ptr(out, torch.int64, "out"), _stream(stream)), "mphf_bucket_u64")
    return out


def mphf_launch_count() -> int:
    return load().mphf_launch_count()


def mphf_lookup_u64(m: MPHF, keys: torch.Tensor, table: torch.Tensor, out: torch.Tensor | None = None,
                    stream=None) -> torch.Tensor:
    """Fused out[i] = table[h(keys[i])]; table is an int32 or int64 tensor of n elements."""
    if table.dtype not in (torch.int32, torch.int64):
        raise ValueError("table must be int32 or int64")
    if out is None:
        out = torch.empty(keys.numel(), dtype=table.dtype, device=keys.device)
    if out.dtype != table.dtype:
        raise ValueError("out must have the table's dtype")
    kp = _dev_ptr(keys, keys.dtype, "keys") if _u64_dtype_ok(keys) else None
    if kp is None:
        raise ValueError("keys must be int64")
    _check(load().mphf_lookup_u64(m.handle, kp, keys.numel(), _dev_ptr(table, table.dtype, "table"),
                                  table.element_size(), _dev_ptr(out, out.dtype, "out"), _stream(stream)),
           "mphf_lookup_u64")
    return out


def mphf_set_l2_fetch_granularity(nbytes: int) -> int:
    """Sets the current context's L2 fetch granularity (0..128 bytes; a hint,
    context-wide); returns the value in force before the call."""
    prev = ctypes.c_int(0)
    _check(load().mphf_set_l2_fetch_granularity(int(nbytes), ctypes.byref(prev)), "mphf_set_l2_fetch_granularity")
    return prev.value


def mphf_build_u64_noalloc(keys: torch.Tensor, params: mphf_params | None = None, stream=None) -> bytes:
    """Builds without allocating device memory (n <= 65536); returns the
    serialized structure, as mphf_serialize would."""
    params = params or mphf_default_params()
    lib = load()
    n = keys.numel()
    cap = 128 + n * 8 + 4096
    need = ctypes.c_size_t()
    buf = ctypes.create_string_buffer(cap)
    rc = lib.mphf_build_u64_noalloc(ctypes.byref(params), _dev_ptr(keys, torch.int64, "keys"), n, buf, cap,
                                    ctypes.byref(need), _stream(stream))
    if rc == MPHF_ERR_ARG and need.value > cap:
        buf = ctypes.create_string_buffer(need.value)
        rc = lib.mphf_build_u64_noalloc(ctypes.byref(params), _dev_ptr(keys, torch.int64, "keys"), n, buf,
                                        need.value, ctypes.byref(need), _stream(stream))
    _check(rc, "mphf_build_u64_noalloc")
    return buf.raw[:need.value]


# ------------------------------------------------------------------ batches
def make_requests(items) -> tuple[ctypes.Array, list]:
    """items: (MPHF, keys tensor, out tensor) or (MPHF, bytes, offsets, out).
    Returns the C array and the tensors it points to (keep them alive)."""
    arr = (mphf_request * max(len(items), 1))()
    keep = []
    for i, it in enumerate(items):
        if len(it) == 3:
            m, keys, out = it
            arr[i] = mphf_request(m.handle.value, _dev_ptr(keys, torch.int64, "keys") if keys.numel() else None,
                                  None, keys.numel(), _dev_ptr(out, torch.int32, "out") if out.numel() else None)
        else:
            m, data, offsets, out = it
            arr[i] = mphf_request(m.handle.value, _dev_ptr(data, torch.uint8, "bytes") if data.numel() else None,
                                  _dev_ptr(offsets, torch.int64, "offsets"), offsets.numel() - 1,
                                  _dev_ptr(out, torch.int32, "out") if out.numel() else None)
        keep.append(it)
    return arr, keep


class Batch:
    """Owns an mphf_batch_t (persistent multi-structure query executor)."""

    def __init__(self, max_requests: int = 1024):
        self._h = ctypes.c_void_p()
        _check(load().mphf_batch_create(max_requests, ctypes.byref(self._h)), "mphf_batch_create")

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mphf_batch_free(h)
            self._h = None

    def run(self, reqs: ctypes.Array, n: int, stream=None):
        _check(load().mphf_batch_run(self._h, reqs, n, _stream(stream)), "mphf_batch_run")

    def set_config(self, keys_per_thread=8, threads=256, blocks_per_sm=4, use_graph=True):
        c = mphf_batch_config(keys_per_thread, threads, blocks_per_sm, int(use_graph))
        _check(load().mphf_batch_set_config(self._h, ctypes.byref(c)), "mphf_batch_set_config")

    def config(self) -> dict:
        c = mphf_batch_config()
        _check(load().mphf_batch_get_config(self._h, ctypes.byref(c)), "mphf_batch_get_config")
        return c.as_dict()

    def autotune(self, reqs: ctypes.Array, n: int, cache_path: str | None = None, stream=None) -> dict:
        c = mphf_batch_config()
        _check(load().mphf_batch_autotune(self._h, reqs, n, _stream(stream),
                                          cache_path.encode() if cache_path else None, ctypes.byref(c)),
               "mphf_batch_autotune")
        return c.as_dict()


# ------------------------------------------------------------------ serving
class Server:
    """Owns an mphf_server_t (continuous-batching serving loop)."""

    def __init__(self, hbm_budget_bytes: int | None = None, max_batch_requests: int | None = None,
                 max_batch_keys: int | None = None, slots: int | None = None):
        lib = load()
        c = mphf_server_config()
        _check(lib.mphf_server_default_config(ctypes.byref(c)), "mphf_server_default_config")
        if hbm_budget_bytes is not None:
            c.hbm_budget_bytes = hbm_budget_bytes
        if max_batch_requests is not None:
            c.max_batch_requests = max_batch_requests
        if max_batch_keys is not None:
            c.max_batch_keys = max_batch_keys
        if slots is not None:
            c.slots = slots
        self._h = ctypes.c_void_p()
        _check(lib.mphf_server_create(ctypes.byref(c), ctypes.byref(self._h)), "mphf_server_create")

    def __del__(self):
        self.close()

    def close(self):
        h = getattr(self, "_h", None)
        if h is not None and h.value:
            load().mphf_server_free(h)
            self._h = None

    def add(self, blob: bytes) -> int:
        sid = ctypes.c_uint32()
        _check(load().mphf_server_add(self._h, blob, len(blob), ctypes.byref(sid)), "mphf_server_add")
        return sid.value

    def remove(self, sid: int):
        _check(load().mphf_server_remove(self._h, sid), "mphf_server_remove")

    @staticmethod
    def request(sid: int, keys: torch.Tensor, out: torch.Tensor, offsets: torch.Tensor | None = None):
        if offsets is None:
            return mphf_server_req(sid, keys.data_ptr() if keys.numel() else None, None, keys.numel(),
                                   out.data_ptr() if out.numel() else None)
        return mphf_server_req(sid, keys.data_ptr() if keys.numel() else None, offsets.data_ptr(),
                               offsets.numel() - 1, out.data_ptr() if out.numel() else None)

    def submit(self, req: mphf_server_req) -> int:
        t = ctypes.c_uint64()
        _check(load().mphf_server_submit(self._h, ctypes.byref(req), ctypes.byref(t)), "mphf_server_submit")
        return t.value

    def replay(self, reqs: list, arrival_us) -> list:
        n = len(reqs)
        arr = (mphf_server_req * max(n, 1))(*reqs)
        at = (ctypes.c_double * max(n, 1))(*[float(x) for x in arrival_us])
        tk = (ctypes.c_uint64 * max(n, 1))()
        _check(load().mphf_server_replay(self._h, arr, at, n, tk), "mphf_server_replay")
        return list(tk)[:n]

    def wait(self, ticket: int, timeout_us: int = 10_000_000) -> int:
        st = ctypes.c_int()
        _check(load().mphf_server_wait(self._h, ticket, timeout_us, ctypes.byref(st)), "mphf_server_wait")
        return st.value

    def drain(self, timeout_us: int = 60_000_000):
        _check(load().mphf_server_drain(self._h, timeout_us), "mphf_server_drain")

    def stats(self, reset: bool = False) -> dict:
        st = mphf_server_stats_t()
        _check(load().mphf_server_stats(self._h, int(reset), ctypes.byref(st)), "mphf_server_stats")
        return st.as_dict()


def mphf_device_view(m: MPHF) -> mphf_view_t:
    """The structure's device view, for kernels that include mphf_device.cuh."""
    v = mphf_view_t()
    _check(load().mphf_device_view(m.handle, ctypes.byref(v)), "mphf_device_view")
    return v
