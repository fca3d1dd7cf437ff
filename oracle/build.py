"""Build the CPU oracle (plain C, FP64) into oracle/_build/liboracle.so.

Test infrastructure: the GPU library never links this.
"""
from __future__ import annotations

import os
import pathlib
import subprocess

HERE = pathlib.Path(__file__).resolve().parent
OUT = HERE / "_build" / "liboracle.so"
SOURCES = [HERE / "lobpcg_oracle.c", HERE / "mlp_oracle.c"]


def build(force: bool = False) -> pathlib.Path:
    srcs = [s for s in SOURCES if s.exists()]
    hdrs = list(HERE.glob("*.h"))
    if OUT.exists() and not force:
        newest = max(p.stat().st_mtime for p in srcs + hdrs)
        if OUT.stat().st_mtime >= newest:
            return OUT
    OUT.parent.mkdir(parents=True, exist_ok=True)
    tmp = OUT.with_suffix(f".tmp{os.getpid()}.so")
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fopenmp", "-ffp-contract=off",
           "-Wall", "-Wextra", "-Wno-unused-parameter", "-o", str(tmp)] + [str(s) for s in srcs] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, OUT)
    return OUT


if __name__ == "__main__":
    print(build(force=True))
