"""In-tree build of the native parts.

libhc.so     : the CUDA library behind include/hc.h (nvcc, sm_103a only)
libhc_check.so: the same sources with -DHC_CHECK (device bounds checks and
               buffer guards, read back by hc_check_status)
libhcgen.so  : the seeded input generator (plain C, gcc)

Translation units compile in parallel into _build/ and link in place next to
this file, so the loaded .so is the in-tree one.
"""
import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD_DIR = os.path.join(PKG, "_build")
HC_LIB = os.path.join(PKG, "libhc.so")
GEN_LIB = os.path.join(PKG, "libhcgen.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
              "-Xcompiler", "-fvisibility=hidden", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale(target, sources):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(s) > t for s in sources)


def _headers():
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE) if f.endswith(".h")]
    return hs


def _run(cmd):
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    if r.returncode != 0:
        raise RuntimeError("command failed: %s\n%s" % (" ".join(cmd), r.stdout))
    return r.stdout


HC_CHECK_LIB = os.path.join(PKG, "libhc_check.so")
VARIANTS = {"normal": (HC_LIB, BUILD_DIR, []),
            "check": (HC_CHECK_LIB, os.path.join(BUILD_DIR, "check"), ["-DHC_CHECK"])}


def build_hc(force=False, verbose=False, extra_flags=(), variants=("normal",)):
    """Compile every csrc/*.cu for sm_103a and link libhc.so (and, when
    asked, libhc_check.so), all translation units of all variants in one
    parallel pool.  Returns the path of the first variant's library."""
    sources = sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith(".cu"))
    headers = _headers()
    nvcc = _nvcc()
    plan, jobs = [], []
    for v in variants:
        lib, bdir, flags = VARIANTS[v]
        os.makedirs(bdir, exist_ok=True)
        objs = []
        for src in sources:
            obj = os.path.join(bdir, os.path.basename(src)[:-3] + ".o")
            objs.append(obj)
            if force or _stale(obj, [src] + headers):
                jobs.append([nvcc] + ARCH + NVCC_FLAGS + flags + list(extra_flags) +
                            ["-c", src, "-o", obj])
        plan.append((lib, objs))
    if jobs:
        with ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(_run, jobs):
                if verbose and out.strip():
                    sys.stdout.write(out)
    for lib, objs in plan:
        if force or jobs or _stale(lib, objs):
            tmp = lib + ".tmp%d" % os.getpid()
            _run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
            os.replace(tmp, lib)
    return plan[0][0]


def build_hc_check(force=False, verbose=False):
    """libhc_check.so alone."""
    return build_hc(force=force, verbose=verbose, variants=("check",))


def build_datagen(force=False):
    src = os.path.join(CSRC, "datagen.c")
    if force or _stale(GEN_LIB, [src]):
        tmp = GEN_LIB + ".tmp%d" % os.getpid()
        _run(["gcc", "-O2", "-std=gnu11", "-fPIC", "-shared", "-ffp-contract=off", "-o", tmp,
              src, "-lm", "-lpthread"])
        os.replace(tmp, GEN_LIB)
    return GEN_LIB


if __name__ == "__main__":
    build_datagen(force="--force" in sys.argv)
    print(build_hc(force="--force" in sys.argv, verbose=True, variants=("normal", "check")))
