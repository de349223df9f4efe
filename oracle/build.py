"""Compile the oracle's C definition into ``oracle/_lib/liboracle.so``.

TEST INFRASTRUCTURE ONLY (see ``oracle/__init__.py``). Plain gcc, OpenMP,
no FMA contraction, no architecture-specific flags, so the x86 build host and
the Arm GPU host produce the same numbers.
"""
from __future__ import annotations

import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))
_SRC = os.path.join(_HERE, "sgemm_ref.c")
_OUT_DIR = os.path.join(_HERE, "_lib")
_OUT = os.path.join(_OUT_DIR, "liboracle.so")


def lib_path() -> str:
    return _OUT


def build(force: bool = False) -> str:
    """Build the shared library if it is missing or older than its source."""
    if (not force and os.path.exists(_OUT)
            and os.path.getmtime(_OUT) >= os.path.getmtime(_SRC)):
        return _OUT
    os.makedirs(_OUT_DIR, exist_ok=True)
    tmp = _OUT + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", "-Wall", "-o", tmp, _SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, _OUT)
    return _OUT
