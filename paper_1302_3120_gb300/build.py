"""Build libcsar.so in-tree with nvcc for sm_103a (no CMake, no torch extension).

Each translation unit under ``csrc/`` is compiled in parallel with
``-gencode arch=compute_103a,code=sm_103a`` and the objects are linked into
``paper_1302_3120_gb300/libcsar.so``.  Objects go to ``_build/`` (git-ignored).
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libcsar.so")
# cuFFT-based comparison build of the ITA iteration (timed by bench.py only; not part of
# libcsar): compare/cufft_ita.cu -> libcsar_cufft.so, linked against libcsar and cuFFT
CHECKED_OUT = os.path.join(HERE, "libcsar_checked.so")
CMP_SRC = os.path.join(HERE, "compare", "cufft_ita.cu")
CMP_OUT = os.path.join(HERE, "libcsar_cufft.so")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
FLAGS += os.environ.get("CSAR_NVCC_EXTRA", "").split()


def nvcc() -> str:
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found (CUDA toolkit required to build libcsar)")
    return path


def sources() -> list[str]:
    return sorted(os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith(".cu"))


def _compile(src: str, verbose: bool, extra=(), bdir: str = BUILD) -> str:
    obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
    cmd = [nvcc(), *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
    if verbose:
        sys.stderr.write(r.stderr)
    return obj


def needs_build() -> bool:
    if not os.path.exists(OUT):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(SRC, f) for f in os.listdir(SRC)]
    deps.append(os.path.join(os.path.dirname(HERE), "include", "csar.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build_compare(force: bool = False) -> str | None:
    """libcsar_cufft.so (the benchmark's cuFFT comparison build); None if it cannot be
    built (the benchmark then reports the comparison as unavailable)."""
    if (not force and os.path.exists(CMP_OUT) and os.path.getmtime(CMP_OUT) >= os.path.getmtime(CMP_SRC)
            and os.path.getmtime(CMP_OUT) >= os.path.getmtime(OUT)):
        return CMP_OUT
    os.makedirs(BUILD, exist_ok=True)
    obj = os.path.join(BUILD, "cufft_ita.o")
    r = subprocess.run([nvcc(), *ARCH, *FLAGS, "-c", CMP_SRC, "-o", obj], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(f"cuFFT comparison build skipped (compile):\n{r.stderr}\n")
        return None
    tmp = CMP_OUT + ".tmp"
    r = subprocess.run([nvcc(), *ARCH, "-shared", "-o", tmp, obj, "-L" + HERE, "-lcsar", "-lcufft",
                        "-lcudart", "-Xlinker", "-rpath=$ORIGIN"], capture_output=True, text=True)
    if r.returncode != 0:
        sys.stderr.write(f"cuFFT comparison build skipped (link):\n{r.stderr}\n")
        return None
    os.replace(tmp, CMP_OUT)
    return CMP_OUT


def build_checked() -> str:
    """libcsar_checked.so: the same library compiled with -DCSAR_CHECKED (global
    indexes of the pass kernels compared with their arrays' extents; an index out of
    range is skipped and reported as CSAR_E_INTERNAL).  Load it by setting
    CSAR_LIB_PATH before importing the binding."""
    return build(force=True, checked=True)


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    out = CHECKED_OUT if checked else OUT
    if not checked and not force and not needs_build():
        return OUT
    bdir = BUILD + ("_checked" if checked else "")
    os.makedirs(bdir, exist_ok=True)
    srcs = sources()
    extra = ["-DCSAR_CHECKED"] if checked else []
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(srcs), os.cpu_count() or 1))) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose, extra, bdir), srcs))
    tmp = out + ".tmp"
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    if not checked:
        build_compare(force=True)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
