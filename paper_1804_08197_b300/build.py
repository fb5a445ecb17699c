"""Builds libsg.so (the C-ABI library) in-tree with nvcc for sm_103a.

    python -m paper_1804_08197_b300.build [--force] [-v]
"""
import os
import subprocess
import sys
import tempfile
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libsg.so")
SOURCES = ["api.cu", "ingest.cu", "tf.cu", "select.cu", "render.cu", "lens.cu", "unet.cu", "lz4.cpp", "container.cpp",
           "stream.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for p in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if p and (os.path.isabs(p) and os.path.exists(p) or not os.path.isabs(p)):
            return p
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "sg.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False, out=None, defines=()):
    """Compiles csrc/*.cu into `out` (default: the in-tree libsg.so): one
    object per source, compiled in parallel, then linked."""
    out = out or LIB
    if out == LIB and not defines and not force and not _stale():
        return LIB
    flags = [*ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-ffp-contract=off",
             "--expt-relaxed-constexpr", "--extended-lambda"]
    flags += [f"-D{d}" for d in defines]
    if verbose:
        flags += ["-Xptxas", "-v"]
    with tempfile.TemporaryDirectory(prefix="sg_build_") as tmp:
        objs = [os.path.join(tmp, os.path.splitext(f)[0] + ".o") for f in SOURCES]

        def compile_one(i):
            subprocess.check_call([_nvcc(), *flags, "-c", os.path.join(CSRC, SOURCES[i]), "-o", objs[i]])

        # the longest compile first
        order = sorted(range(len(SOURCES)), key=lambda i: os.path.getsize(os.path.join(CSRC, SOURCES[i])),
                       reverse=True)
        with ThreadPoolExecutor(max_workers=max(1, min(len(SOURCES), os.cpu_count() or 1))) as ex:
            for f in [ex.submit(compile_one, i) for i in order]:
                f.result()
        subprocess.check_call([_nvcc(), *ARCH, "-shared", "-o", out + ".tmp", *objs])
    os.replace(out + ".tmp", out)
    return out


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="-v" in sys.argv)
    print(LIB)
