"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liboracle.so.

-ffp-contract=off keeps x86-64 and aarch64 results identical (no fused
multiply-add contraction); OpenMP parallelises the z-plane loops only.
"""
import os
import subprocess
import sys

_HERE = os.path.dirname(os.path.abspath(__file__))


def build_oracle(force: bool = False) -> str:
    srcs = [os.path.join(_HERE, f) for f in ("fdtd_oracle.c", "fdtd_oracle_complex.c")]
    out = os.path.join(_HERE, "liboracle.so")
    if not force and os.path.exists(out) and all(os.path.getmtime(out) >= os.path.getmtime(s) for s in srcs):
        return out
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-fopenmp"] + srcs + ["-o", tmp, "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle(force="--force" in sys.argv))
