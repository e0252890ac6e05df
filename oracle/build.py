"""Compiles the CPU oracle (plain C) into a shared library with gcc.

Test infrastructure: nothing in the GPU library calls this.  ``mutant`` builds
a copy with one planted mistake (ORACLE_MUTANT) into a separate file; the tests
use those copies to show that the oracle's pins catch such mistakes.
"""
from __future__ import annotations

import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "oracle.c")
OUT_DIR = os.path.join(HERE, "_build")


def lib_path(mutant: int = 0, out_dir: str | None = None) -> str:
    name = "liboracle.so" if not mutant else f"liboracle_mutant{mutant}.so"
    return os.path.join(out_dir or OUT_DIR, name)


def build(force: bool = False, mutant: int = 0, out_dir: str | None = None) -> str:
    out = lib_path(mutant, out_dir)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-Wall", "-Wextra",
           f"-DORACLE_MUTANT={int(mutant)}", SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


CPU_SRC = os.path.join(HERE, "cpu_baselines.cpp")


def cpu_lib_path(out_dir: str | None = None) -> str:
    return os.path.join(out_dir or OUT_DIR, "libcpu_baselines.so")


def build_cpu(force: bool = False, out_dir: str | None = None) -> str:
    """The benchmark's CPU comparison sorts (std::sort on one core and on
    every core), built with g++."""
    out = cpu_lib_path(out_dir)
    if not force and os.path.exists(out) and os.path.getmtime(out) >= os.path.getmtime(CPU_SRC):
        return out
    os.makedirs(os.path.dirname(out), exist_ok=True)
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-Wall", "-Wextra", CPU_SRC, "-o", tmp]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
    print(build_cpu(force="--force" in sys.argv))
