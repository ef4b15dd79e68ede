"""Builds librecoil.so in-tree for sm_103a (nvcc cross-compiles without a GPU)."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "librecoil.so")
SOURCES = ["decode_kernels.cu", "plan.cpp", "host_codec.cpp", "tune.cpp", "serve.cpp", "serve_kernels.cu", "pipeline.cpp",
           "serialize.cpp", "noalloc.cu"]
HEADERS = ["recoil_internal.h", "device_types.h"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, out: str = LIB, defines=()) -> str:
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    deps = srcs + [os.path.join(CSRC, h) for h in HEADERS] + [os.path.join(ROOT, "include", "recoil.h")]
    if not force and not _stale(out, deps):
        return out
    nvcc = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
    tmp = out + f".tmp{os.getpid()}"
    cmd = [nvcc, "-O3", "-std=c++17", *ARCH, "-lineinfo", "-Xcompiler", "-fPIC,-O3,-Wall",
           "-shared", "-cudart", "shared", "-I", os.path.join(ROOT, "include"), "-I", CSRC,
           *[f"-D{d}" for d in defines], *srcs, "-o", tmp]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
        print(" ".join(cmd), file=sys.stderr)
    subprocess.check_call(cmd)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
