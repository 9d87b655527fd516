"""Build the CUDA/C++ library libjet.so in-tree for sm_103a (B300).

nvcc compiles the .cu kernels (-gencode arch=compute_103a,code=sm_103a), g++
the host planner and C ABI; the result links the CUDA runtime statically and
needs no other CUDA library at run time.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
SO = os.path.join(HERE, "libjet.so")
CUDA = os.environ.get("CUDA_HOME", "/usr/local/cuda")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
INC = ["-I", os.path.join(ROOT, "include"), "-I", SRC, "-I", os.path.join(CUDA, "include")]


def _sources():
    return sorted(f for f in os.listdir(SRC) if f.endswith((".cu", ".cpp")))


def _headers_mtime():
    hs = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    hs.append(os.path.join(ROOT, "include", "jet.h"))
    return max(os.path.getmtime(h) for h in hs)


def _compile(src, verbose=False):
    out = os.path.join(OBJ, src + ".o")
    path = os.path.join(SRC, src)
    if os.path.exists(out) and os.path.getmtime(out) >= max(os.path.getmtime(path), _headers_mtime()):
        return out
    if src.endswith(".cu"):
        cmd = [os.path.join(CUDA, "bin", "nvcc"), "-O3", "-std=c++17", *ARCH, "-lineinfo",
               "-Xcompiler", "-fPIC", "-Xptxas", "-v" if verbose else "-O3", *INC, "-c", path, "-o", out]
    else:
        cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-Wall", "-Wno-unused-function", *INC, "-c", path, "-o", out]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"compile failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    if verbose and r.stderr:
        sys.stderr.write(r.stderr)
    return out


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    if force:
        for f in os.listdir(OBJ):
            os.remove(os.path.join(OBJ, f))
    with cf.ThreadPoolExecutor(max_workers=min(8, os.cpu_count() or 1)) as ex:
        objs = list(ex.map(lambda s: _compile(s, verbose), _sources()))
    if os.path.exists(SO) and os.path.getmtime(SO) >= max(os.path.getmtime(o) for o in objs):
        return SO
    tmp = SO + f".tmp{os.getpid()}"
    cmd = [os.path.join(CUDA, "bin", "nvcc"), "-shared", *ARCH, "-Xcompiler", "-fPIC",
           "--cudart", "static", "-Xlinker", "--exclude-libs,ALL", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, SO)
    return SO


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
