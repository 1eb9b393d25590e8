"""Build the CUDA library libbdm_gb300.so in-tree for sm_103a (GB300).

Each translation unit is compiled by nvcc in parallel, then linked into one
shared library under paper_2301_06984_gb300/_build/.  No torch types cross
the C ABI; the library links the CUDA runtime only.

build(variant="check") builds libbdm_gb300_check.so with -DBDM_CHECK: every
index a kernel derives from device data is range-checked, and a failed check
is reported through the device error word (source line included) instead of
touching memory out of range.  Select it with BDM_LIBRARY=<path>.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libbdm_gb300.so")
SOURCES = ["engine.cu", "grid.cu", "force.cu", "noalloc.cu", "params.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "-I", CSRC, "-I", INCLUDE]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


LIB_CHECK = os.path.join(OUT_DIR, "check", "libbdm_gb300_check.so")


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False, variant: str = "") -> str:
    out_dir = os.path.join(OUT_DIR, variant) if variant else OUT_DIR
    lib = LIB_CHECK if variant == "check" else LIB
    extra = ["-DBDM_CHECK"] if variant == "check" else []
    os.makedirs(out_dir, exist_ok=True)
    headers = [os.path.join(CSRC, "bdm_internal.cuh"), os.path.join(INCLUDE, "bdm.h")]
    objs = []
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(out_dir, src.replace(".cu", ".o"))
        objs.append(o)
        if force or _stale(o, [s] + headers):
            cmd = [_nvcc()] + ARCH + NVCC_FLAGS + extra + (["-Xptxas", "-v"] if ptxas_info else []) + \
                  ["-c", s, "-o", o]
            jobs.append(cmd)
    with cf.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(lambda c: subprocess.run(c, capture_output=True, text=True), jobs))
    for cmd, r in zip(jobs, results):
        if verbose or ptxas_info or r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed: %s" % " ".join(cmd))
    if force or jobs or _stale(lib, objs):
        tmp = lib + ".tmp.%d" % os.getpid()
        cmd = [_nvcc()] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed")
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv,
                variant="check" if "--check" in sys.argv else ""))
