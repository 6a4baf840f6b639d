"""Compile the FP64 CPU oracle (test infrastructure) into oracle/liblbm_oracle.so.

Plain gcc, no fused multiply-add (-ffp-contract=off) so that the oracle gives
the same bits on x86_64 and aarch64 hosts; OpenMP only splits the per-cell
loop of a time step, which does not change any result.
"""
import os
import pathlib
import subprocess

HERE = pathlib.Path(__file__).resolve().parent
SRCS = [HERE / "lbm_oracle.c", HERE / "lbm3d_oracle.c"]
LIB = HERE / "liblbm_oracle.so"


def build(force: bool = False) -> pathlib.Path:
    if not force and LIB.exists() and all(LIB.stat().st_mtime >= s.stat().st_mtime for s in SRCS):
        return LIB
    cc = os.environ.get("CC", "gcc")
    tmp = LIB.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [cc, "-O2", "-std=c11", "-Wall", "-ffp-contract=off", "-fno-fast-math", "-fopenmp",
           "-fPIC", "-shared", *[str(s) for s in SRCS], "-o", str(tmp), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
