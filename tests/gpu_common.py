"""Shared helpers of the GPU tests (structures are built by the oracle, so no
expected value comes from the CUDA path)."""
from __future__ import annotations

import functools

import numpy as np
import pytest
import torch

from oracle import oracle as O
from paper_2502_15539_gb300 import workloads as W


def need_gpu():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2502_15539_gb300 import build_ext, native
    build_ext.build()
    native.load()
    return native


@functools.lru_cache(maxsize=None)
def oracle_structure(n: int, key_seed: int = 0, **params) -> tuple[O.OracleMPHF, bytes]:
    keys = W.as_uint64_numpy(W.u64_keys(n, key_seed))
    threads = 16 if n >= 10**6 else 1
    m = O.OracleMPHF.build_u64(keys, threads=threads, **params)
    return m, m.serialize()


def u32(t: torch.Tensor) -> np.ndarray:
    return t.detach().cpu().numpy().view(np.uint32)


def oracle_values_of(N, m, keys=None, data=None, offsets=None) -> np.ndarray:
    """The oracle's evaluation of a library structure: its serialized bytes
    are loaded by the oracle's own reader and queried one key at a time, so a
    GPU-built structure is checked against the formula, not only for being a
    bijection (Sec. 3.2)."""
    ref = O.OracleMPHF.deserialize(N.mphf_serialize(m))
    if keys is not None:
        k = W.as_uint64_numpy(keys)
        return ref.query_u64(k, threads=16 if len(k) >= 10**5 else 1)
    d = data.detach().cpu().numpy()
    o = offsets.detach().cpu().numpy().astype(np.uint64)
    return ref.query_bytes(d, o, threads=16 if len(o) > 10**5 else 1)
