"""Builds libdbmp.so (sm_103a) in-tree with nvcc: one object per .cu, compiled in
parallel, linked with the shared CUDA runtime, and the same sources with device-side
index checks (-DDBMP_CHECKED=1) as libdbmp_checked.so.  Output:
paper_2602_22625_gb300/_lib/."""
import concurrent.futures as cf
import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_lib")
LIB = os.path.join(OUT, "libdbmp.so")
LIB_CHECKED = os.path.join(OUT, "libdbmp_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              "--expt-relaxed-constexpr", "-I", os.path.join(ROOT, "include")]


def nvcc() -> str:
    p = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(p):
        raise RuntimeError("nvcc not found")
    return p


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")))


def _deps():
    return sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        [os.path.join(ROOT, "include", "dbmp.h"), __file__]


def up_to_date() -> bool:
    for lib in (LIB, LIB_CHECKED):
        if not os.path.exists(lib):
            return False
        t = os.path.getmtime(lib)
        if any(os.path.getmtime(d) > t for d in _deps()):
            return False
    return True


def build(force: bool = False, verbose_ptxas: bool = False) -> str:
    if not force and up_to_date():
        return LIB
    cc = nvcc()
    extra = ["-Xptxas", "-v"] if verbose_ptxas else []
    variants = (("obj", [], LIB), ("obj_checked", ["-DDBMP_CHECKED=1"], LIB_CHECKED))
    for sub, _, _ in variants:
        os.makedirs(os.path.join(OUT, sub), exist_ok=True)

    def compile_one(job):
        src, sub, flags = job
        obj = os.path.join(OUT, sub, os.path.basename(src) + ".o")
        cmd = [cc, *ARCH, *NVCC_FLAGS, *flags, *(extra if not flags else []), "-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        return obj, r.stderr

    jobs = [(src, sub, flags) for sub, flags, _ in variants for src in sources()]
    with cf.ThreadPoolExecutor(max_workers=min(16, os.cpu_count() or 4)) as ex:
        results = list(ex.map(compile_one, jobs))
    if verbose_ptxas:
        for (_, sub, _), (_, err) in zip(jobs, results):
            if sub == "obj":
                sys.stderr.write(err)
    for sub, _, lib in variants:
        objs = [o for (_, s, _), (o, _) in zip(jobs, results) if s == sub]
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [cc, *ARCH, "-shared", "-cudart", "shared", "-o", tmp, *objs]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
