"""Runs a snippet in a child Python process with the NVTX recorder
(tests/nvtx_record.c) injected, and returns the recorded range lines."""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)


def build_recorder(out_dir):
    cuda = os.environ.get("CUDA_HOME", "/usr/local/cuda")
    so = os.path.join(str(out_dir), "libnvtx_record.so")
    subprocess.run(["gcc", "-O2", "-fPIC", "-shared", "-I" + os.path.join(cuda, "include"),
                    "-o", so, os.path.join(HERE, "nvtx_record.c"), "-lpthread"], check=True)
    return so


def record(code, out_dir, timeout=600):
    so = build_recorder(out_dir)
    log = os.path.join(str(out_dir), "nvtx.log")
    env = dict(os.environ, NVTX_INJECTION64_PATH=so, HC_NVTX_LOG=log)
    r = subprocess.run([sys.executable, "-c", code], env=env, cwd=ROOT, timeout=timeout,
                       stdout=subprocess.PIPE, stderr=subprocess.STDOUT, text=True)
    assert r.returncode == 0, r.stdout
    return open(log).read().splitlines() if os.path.exists(log) else []


def balanced(lines):
    """True when every pop closes an open range and none stays open."""
    depth = 0
    for ln in lines:
        depth += 1 if ln.startswith("push ") else -1
        if depth < 0:
            return False
    return depth == 0
