"""Builds the solver's shared library in-tree: paper_2202_10313_gb300/libaderlts.so.

Host set-up (C++17, g++) and CUDA kernels (nvcc, sm_103a only) are compiled as separate
translation units in parallel and linked with nvcc. Before them, a small host program
(gen_sparse.cpp, built with the library's host basis code) writes the sparse operator
products of the predict kernel into _build/sparse_ops.cuh. Usage: ``python -m
paper_2202_10313_gb300.build`` or ``build()``.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libaderlts.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
HOST_SOURCES = ["host_basis.cpp", "host_mesh.cpp", "host_setup.cpp", "host_partition.cpp"]
CUDA_SOURCES = ["api.cu", "kernels_o3.cu", "kernels_o4.cu", "kernels_o5.cu", "energy_noalloc.cu", "peaks.cu"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("build step failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


def _stale(obj, srcs):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(s) > t for s in srcs)


def _generate_sparse_ops():
    """Builds and runs the generator of the sparse operator products (gen_sparse.cpp with the
    library's own host basis code) -> _build/sparse_ops.cuh, when its inputs changed."""
    gen_src = [os.path.join(SRC, f) for f in ("gen_sparse.cpp", "host_basis.cpp", "host.h")]
    exe = os.path.join(OUT_DIR, "gen_sparse")
    out = os.path.join(OUT_DIR, "sparse_ops.cuh")
    if _stale(exe, gen_src):
        _run(["g++", "-std=c++17", "-O2", "-Wall", gen_src[0], gen_src[1], "-o", exe])
    if _stale(out, [exe]):
        _run([exe, out + ".tmp"])
        os.replace(out + ".tmp", out)
    return out


def build(verbose=False, ptxas_info=False):
    os.makedirs(OUT_DIR, exist_ok=True)
    headers = [os.path.join(SRC, f) for f in os.listdir(SRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(HERE, "..", "include", "ader_lts.h"))
    headers.append(_generate_sparse_ops())
    jobs = []
    objs = []
    for f in HOST_SOURCES:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            jobs.append(["g++", "-std=c++17", "-O2", "-fPIC", "-Wall", "-c", src, "-o", obj])
    for f in CUDA_SOURCES:
        src = os.path.join(SRC, f)
        obj = os.path.join(OUT_DIR, f + ".o")
        objs.append(obj)
        if _stale(obj, [src] + headers):
            cmd = [_nvcc(), "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-I", OUT_DIR,
                   "-c", src, "-o", obj] + ARCH
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append(cmd)
    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(_run, jobs):
            if verbose and out.strip():
                print(out)
    if jobs or not os.path.exists(LIB):
        _run([_nvcc(), "-shared", "-o", LIB] + objs + ARCH + ["-lcudart"])
    return LIB


if __name__ == "__main__":
    build(verbose=True, ptxas_info="-v" in sys.argv)
    print(LIB)
