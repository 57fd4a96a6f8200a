"""Compile the plain C programs of the tests against include/pgm.h and
libpgm.so (strict C99, warnings as errors; the CUDA runtime's own headers
are included as system headers)."""
import os
import shutil
import subprocess

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def cuda_home():
    from paper_1704_03217_gb300 import build
    nvcc = build.NVCC if os.path.isabs(build.NVCC) else shutil.which(build.NVCC)
    return os.path.dirname(os.path.dirname(os.path.realpath(nvcc))) if nvcc else None


def compile_c(src, exe, cudart=False):
    """Build tests/<src> into `exe`; returns (ok, compiler output)."""
    from paper_1704_03217_gb300 import build
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        return None, "no C compiler"
    libdir = os.path.dirname(build.build())
    cmd = [cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic",
           "-I", os.path.join(ROOT, "include"), os.path.join(ROOT, "tests", src),
           "-L", libdir, "-lpgm", "-Wl,-rpath," + libdir, "-o", exe]
    if cudart:
        home = cuda_home()
        if home is None:
            return None, "no CUDA toolkit"
        lib = os.path.join(home, "lib64")
        cmd[1:1] = ["-isystem", os.path.join(home, "include")]
        cmd += ["-L", lib, "-lcudart", "-Wl,-rpath," + lib]
    r = subprocess.run(cmd, capture_output=True, text=True)
    return r.returncode == 0, r.stdout + r.stderr
