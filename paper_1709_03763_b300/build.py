"""Build libsurfcorr.so in-tree: nvcc for sm_103a (B300), no JIT at import time.

Each source compiles to its own object (in parallel, under _build/), then one link
step makes the shared library; an object is rebuilt when its source, a header or the
flags are newer than it.
"""
import glob
import hashlib
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libsurfcorr.so")
OBJ_DIR = os.path.join(HERE, "_build")

NVCC_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-O3", "-lineinfo", "-std=c++17",
              "-Xcompiler", "-fPIC", "-Xcompiler", "-O2", "-Xptxas", "-v"]
LINK_FLAGS = ["-gencode", "arch=compute_103a,code=sm_103a", "-cudart", "shared", "-shared"]


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def headers():
    return glob.glob(os.path.join(CSRC, "*.cuh")) + [os.path.join(INCLUDE, "surfcorr.h")]


def _flag_tag() -> str:
    return hashlib.sha1(" ".join(NVCC_FLAGS).encode()).hexdigest()[:8]


def _obj(src: str) -> str:
    return os.path.join(OBJ_DIR, os.path.basename(src) + "." + _flag_tag() + ".o")


def stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(f) > t for f in sources() + headers())


def _compile(nvcc: str, src: str):
    out = _obj(src)
    cmd = [nvcc, *NVCC_FLAGS, "-I", INCLUDE, "-c", "-o", out + ".tmp", src]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode == 0:
        os.replace(out + ".tmp", out)
    return src, r


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not stale():
        return LIB
    nvcc = os.environ.get("NVCC", "nvcc")
    os.makedirs(OBJ_DIR, exist_ok=True)
    newest_header = max(os.path.getmtime(h) for h in headers())
    todo = [s for s in sources() if force or not os.path.exists(_obj(s)) or
            os.path.getmtime(_obj(s)) < max(os.path.getmtime(s), newest_header)]
    failed = []
    with ThreadPoolExecutor(max_workers=max(1, min(len(todo) or 1, os.cpu_count() or 1))) as ex:
        for src, r in ex.map(lambda s: _compile(nvcc, s), todo):
            if verbose or r.returncode != 0:
                sys.stderr.write(r.stdout + r.stderr)
            if r.returncode != 0:
                failed.append(os.path.basename(src))
    if failed:
        raise RuntimeError("nvcc failed building libsurfcorr.so: " + ", ".join(failed))
    cmd = [nvcc, *LINK_FLAGS, "-o", LIB + ".tmp", *[_obj(s) for s in sources()]]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if verbose or r.returncode != 0:
        sys.stderr.write(r.stdout + r.stderr)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed linking libsurfcorr.so")
    os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
