"""Builds the caller kernels of tests/device_api_caller.cu against the public
device header, the way an application links its own kernels."""
from __future__ import annotations

import functools
import os
import shutil
import subprocess
import tempfile

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CALLER = os.path.join(ROOT, "tests", "device_api_caller.cu")


def nvcc() -> str | None:
    found = shutil.which("nvcc")
    if found:
        return found
    default = "/usr/local/cuda/bin/nvcc"
    return default if os.path.exists(default) else None


def compile_caller(out: str, shared: bool) -> None:
    cmd = [nvcc(), "-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-std=c++17",
           "-I", os.path.join(ROOT, "include"), CALLER, "-o", out]
    cmd[1:1] = ["-shared", "-Xcompiler", "-fPIC"] if shared else ["-c"]
    subprocess.run(cmd, check=True, capture_output=True, text=True)


@functools.lru_cache(maxsize=None)
def caller_library() -> str:
    path = os.path.join(tempfile.mkdtemp(prefix="mphf_caller_"), "libmphf_caller.so")
    compile_caller(path, shared=True)
    return path
