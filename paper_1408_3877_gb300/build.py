"""Build the CUDA library libfestung.so in-tree (nvcc, sm_103a only).

Each translation unit is compiled in parallel into ``_build/`` and linked into
``paper_1408_3877_gb300/libfestung.so``.  The CUDA runtime is linked statically, so
the library only needs the NVIDIA driver at run time.
"""
import os
import shutil
import subprocess
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(PKG, "libfestung.so")
SOURCES = ["tables.cpp", "mesh.cpp", "festung.cu", "batch.cu", "apply_f64.cu", "apply_f32.cu", "apply_f32_kr.cu", "apply_df.cu", "apply_bf16.cu", "bicg_persist.cu", "warmstart.cu", "noalloc.cu", "mlp.cu", "peak.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found")
    return path


def flags(extra=()):
    return ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC,-O3", "-I" + os.path.join(ROOT, "include"),
            "-I" + BUILD, *ARCH, *extra]


def _compile(src, extra):
    obj = os.path.join(BUILD, os.path.basename(src) + ".o")
    cmd = [nvcc(), *flags(extra), "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr[-8000:]))
    return obj, r.stderr


def gen_tables():
    """Compile and run gen_tables (host code: the library's own table builder) to write the
    FP32 reference tables as device constants into _build/festung_tables_gen.h."""
    exe = os.path.join(BUILD, "gen_tables")
    cmd = [nvcc(), "-O2", "-std=c++17", "-I" + os.path.join(ROOT, "include"), "-x", "cu",
           os.path.join(CSRC, "gen_tables.cpp"), "-x", "cu", os.path.join(CSRC, "tables.cpp"), "-o", exe]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gen_tables build failed:\n%s\n%s" % (" ".join(cmd), r.stderr[-4000:]))
    out = os.path.join(BUILD, "festung_tables_gen.h")
    r = subprocess.run([exe, out], capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("gen_tables failed:\n%s" % r.stderr[-4000:])
    return out


def build(verbose=False, extra=()):
    os.makedirs(BUILD, exist_ok=True)
    gen_tables()
    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda s: _compile(s, extra), SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            if log.strip():
                print(log)
    tmp = LIB + ".tmp"
    cmd = [nvcc(), "-shared", *ARCH, "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-4000:])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(verbose=True, extra=sys.argv[1:]))
