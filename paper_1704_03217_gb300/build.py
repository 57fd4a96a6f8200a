"""Build libpgm.so in-tree with nvcc for sm_103a (GB300).

Each translation unit is compiled in parallel, then linked into
paper_1704_03217_gb300/_build/libpgm.so.  No torch extension machinery: the
library has a plain C ABI (include/pgm.h).  build(checked=True) makes
libpgm_checked.so, the same sources with device index checks (-DPGM_CHECKED)
that report PGM_ERR_DEVICE_BOUNDS; PGM_CHECKED=1 in the environment makes the
binding load it.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libpgm.so")
LIB_CHECKED = os.path.join(OUT, "libpgm_checked.so")
SOURCES = ["abi.cu", "pyramid.cu", "match.cu", "pm_row.cu", "init_tile.cu", "init_tc.cu", "filter.cu",
           "filter_noalloc.cu", "interp.cu"]
GENCODE = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
if not os.path.exists(NVCC):
    NVCC = "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "pgm.h"))
    return files


def build(force: bool = False, verbose: bool = False, checked: bool = False) -> str:
    os.makedirs(OUT, exist_ok=True)
    lib = LIB_CHECKED if checked else LIB
    if not force and os.path.exists(lib):
        if os.path.getmtime(lib) >= max(os.path.getmtime(f) for f in _deps()):
            return lib
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
             "-I", os.path.join(ROOT, "include")] + GENCODE
    if checked:
        flags += ["-DPGM_CHECKED"]
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(OUT, src.replace(".cu", "_checked.o" if checked else ".o"))
        cmd = [NVCC, "-c", os.path.join(CSRC, src), "-o", obj] + flags
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed on %s:\n%s%s" % (src, r.stdout, r.stderr))
        if verbose:
            sys.stderr.write(r.stdout + r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = lib + ".tmp%d" % os.getpid()
    cmd = [NVCC, "-shared", "-o", tmp] + objs + GENCODE + ["-lcudart", "-ldl"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                checked="--checked" in sys.argv))
