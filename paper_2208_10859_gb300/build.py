"""Build libwv.so from csrc/*.cu for GB300 (sm_103a) with nvcc, in tree.

Each translation unit is compiled in parallel, then linked into
paper_2208_10859_gb300/_build/libwv.so.  Rebuilds only when a source or header
is newer than the library.
"""
from __future__ import annotations

import glob
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libwv.so")
# the WV_CHECKED build (device bounds checks that record WV_ERR_DEVICE and
# skip the access): a separate library the binding loads when the
# environment variable WV_CHECKED is 1
BUILD_CHECKED = os.path.join(HERE, "_build_checked")
LIB_CHECKED = os.path.join(BUILD_CHECKED, "libwv_checked.so")
# host code under AddressSanitizer and UndefinedBehaviorSanitizer (device
# code unchanged): loaded when the environment variable WV_SANITIZE is 1,
# with the sanitizer runtimes preloaded
BUILD_SAN = os.path.join(HERE, "_build_san")
LIB_SAN = os.path.join(BUILD_SAN, "libwv_san.so")
SAN_FLAGS = ["-Xcompiler=-fsanitize=address", "-Xcompiler=-fsanitize=undefined",
             "-Xcompiler=-fno-sanitize-recover=undefined", "-Xcompiler=-fno-omit-frame-pointer"]
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O2",
              "--expt-relaxed-constexpr", "-I", INCLUDE]


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def sources() -> list[str]:
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _stale(lib: str) -> bool:
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra_flags: list[str] | None = None,
          checked: bool = False, sanitize: bool = False) -> str:
    """Compile and link libwv.so (checked: libwv_checked.so with WV_CHECKED=1;
    sanitize: libwv_san.so, host code under ASan and UBSan); returns its path."""
    lib, out_dir = (LIB_CHECKED, BUILD_CHECKED) if checked else (LIB_SAN, BUILD_SAN) if sanitize else (LIB, BUILD)
    if not force and not _stale(lib):
        return lib
    os.makedirs(out_dir, exist_ok=True)
    nvcc = _nvcc()
    flags = ARCH + NVCC_FLAGS + list(extra_flags or []) + (["-DWV_CHECKED=1"] if checked else []) + \
        (SAN_FLAGS if sanitize else [])

    def compile_one(src: str) -> str:
        obj = os.path.join(out_dir, os.path.basename(src)[:-3] + ".o")
        cmd = [nvcc, *flags, "-c", src, "-o", obj]
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed on {src}:\n{r.stdout}\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr, file=sys.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 4)) as ex:
        objs = list(ex.map(compile_one, sources()))
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, checked="--checked" in sys.argv,
                sanitize="--sanitize" in sys.argv))
