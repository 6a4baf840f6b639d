"""In-tree build of the CUDA library (sm_103a) with nvcc.

One shared object, paper_1303_0107_gb300/_lib/liblbm_gb300.so, compiled from
every csrc/*.cu in one parallel nvcc call, CUDA runtime linked statically.
"""
import os
import pathlib
import subprocess

PKG = pathlib.Path(__file__).resolve().parent
ROOT = PKG.parent
CSRC = PKG / "csrc"
OUT_DIR = PKG / "_lib"
LIB = OUT_DIR / "liblbm_gb300.so"
# bounds-checked variant (every kernel access checked; for debugging only)
LIB_CHECKED = OUT_DIR / "liblbm_gb300_checked.so"
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def sources():
    return sorted(CSRC.glob("*.cu"))


def _stale(lib=LIB) -> bool:
    if not lib.exists():
        return True
    t = lib.stat().st_mtime
    deps = list(sources()) + list(CSRC.glob("*.h")) + list(CSRC.glob("*.cuh")) + list((ROOT / "include").glob("*.h"))
    return any(p.stat().st_mtime > t for p in deps)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> pathlib.Path:
    lib = LIB_CHECKED if checked else LIB
    if not force and not _stale(lib):
        return lib
    OUT_DIR.mkdir(exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    tmp = lib.with_suffix(f".so.tmp{os.getpid()}")
    cmd = [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2", "-shared",
           "-cudart", "static", "--threads", str(min(8, os.cpu_count() or 1)),
           "-I", str(ROOT / "include"), *[str(s) for s in sources()], "-o", str(tmp)]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    if checked:
        cmd.insert(1, "-DLBM_CHECK_BOUNDS")
    subprocess.run(cmd, check=True)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True, verbose=True))
