"""Build the CUDA library in-tree: paper_2605_21398_gb300/_build/libdock.so.

Each translation unit is compiled separately (in parallel) for sm_103a only,
then linked with the static CUDA runtime.  k_object.cu is compiled with
-fmad=false (its FP64 expressions must round exactly as written); the host
runtime with -ffp-contract=off for the same reason.
"""
import concurrent.futures
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libdock.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
INC = os.path.join(os.path.dirname(HERE), "include")


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _units():
    nv = _nvcc()
    cuda_home = os.path.dirname(os.path.dirname(nv))
    common = [nv, "-c", "-O3", "-lineinfo", "-std=c++17", "--expt-relaxed-constexpr", "-Xcompiler", "-fPIC",
              "-I", INC] + ARCH
    units = []
    for src in sorted(os.listdir(CSRC)):
        path = os.path.join(CSRC, src)
        obj = os.path.join(OUT, src + ".o")
        if src.endswith(".cu"):
            extra = ["-fmad=false"] if src == "k_object.cu" else []
            units.append((path, obj, common + extra + ["-o", obj, path]))
        elif src.endswith(".cpp"):
            cmd = ["g++", "-c", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fvisibility=hidden",
                   "-I", os.path.join(cuda_home, "include"), "-I", INC, "-o", obj, path]
            units.append((path, obj, cmd))
    return units


def build(force=False, verbose=False):
    os.makedirs(OUT, exist_ok=True)
    units = _units()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INC, "dock.h"))
    newest_hdr = max(os.path.getmtime(h) for h in headers)
    todo = [u for u in units if force or not os.path.exists(u[1]) or
            os.path.getmtime(u[1]) < max(os.path.getmtime(u[0]), newest_hdr)]

    def run(u):
        r = subprocess.run(u[2], capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed: %s\n%s%s" % (" ".join(u[2]), r.stdout, r.stderr))
        if verbose and r.stderr:
            print(r.stderr)
        return u[1]

    with concurrent.futures.ThreadPoolExecutor(max_workers=min(8, max(1, len(todo)))) as ex:
        list(ex.map(run, todo))
    objs = [u[1] for u in units]
    if todo or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [_nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-Xcompiler", "-fPIC", "--cudart=static",
                                                            "-lpthread", "-ldl", "-lrt"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed: %s\n%s%s" % (" ".join(cmd), r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose=True))
