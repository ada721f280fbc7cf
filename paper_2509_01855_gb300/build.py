"""Build libbirkhoff.so in-tree with nvcc for sm_103a (GB300).

Usage: python -m paper_2509_01855_gb300.build   (or call build()).
Translation units compile in parallel; the shared library lands next to this file.
"""
import concurrent.futures
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libbirkhoff.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
         "--expt-relaxed-constexpr", "-DNDEBUG"]
SOURCES = ["bk_birkhoff.cu", "bk_birkhoff_f64.cu", "bk_birkhoff_f32.cu", "bk_birkhoff_df.cu", "bk_dense.cu",
           "bk_kkt.cu", "bk_krylov.cu", "bk_newton.cu"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.sep not in c or os.path.exists(c)):
            return c
    return "nvcc"


def _needs(obj, src, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in [src] + deps)


def build(verbose=False, force=False):
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    headers.append(os.path.join(os.path.dirname(HERE), "include", "birkhoff.h"))
    jobs = []
    objs = []
    for src in [f for f in SOURCES if os.path.exists(os.path.join(CSRC, f))]:
        sp = os.path.join(CSRC, src)
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        deps = headers + ([os.path.join(CSRC, "bk_birkhoff.cu")]
                          if src in ("bk_birkhoff_f64.cu", "bk_birkhoff_f32.cu", "bk_birkhoff_df.cu") else [])
        if force or _needs(obj, sp, deps):
            jobs.append([nvcc] + ARCH + FLAGS + ["-c", sp, "-o", obj])

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    with concurrent.futures.ThreadPoolExecutor(max_workers=max(1, len(jobs))) as ex:
        for cmd, r in ex.map(run, jobs):
            if verbose or r.returncode != 0:
                sys.stderr.write(" ".join(cmd) + "\n" + r.stdout + r.stderr)
            if r.returncode != 0:
                raise RuntimeError("nvcc failed on " + cmd[-3])
    if force or jobs or not os.path.exists(OUT):
        cmd = [nvcc] + ARCH + ["-shared", "-o", OUT] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link of libbirkhoff.so failed")
    return OUT


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv, force="-f" in sys.argv))
