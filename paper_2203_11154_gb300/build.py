"""Builds libparadiag.so (the CUDA kernels and the C ABI of include/paradiag.h) in-tree.

nvcc compiles each translation unit for sm_103a only, in parallel; the shared library
links the CUDA runtime statically, so it needs nothing from PyTorch.
"""
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD_DIR, "libparadiag.so")
CU_SOURCES = ["mg_kernels.cu", "fused_kernels.cu", "stream_kernels.cu", "transforms.cu",
              "tc_transforms.cu", "host.cu", "static_residual.cu", "shift_refine.cu",
              "residual_ws.cu", "fft_transforms.cu"]
CPP_SOURCES = ["setup.cpp", "eig.cpp"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libparadiag.so")


def _sources():
    return [os.path.join(CSRC, f) for f in CU_SOURCES + CPP_SOURCES] + \
        [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))] + \
        [os.path.join(HERE, "..", "include", "paradiag.h")]


def up_to_date():
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(s) <= t for s in _sources())


def build(force=False, verbose=False):
    if not force and up_to_date():
        return LIB
    nvcc = _nvcc()
    os.makedirs(BUILD_DIR, exist_ok=True)
    jobs = []
    objs = []
    for f in CU_SOURCES + CPP_SOURCES:
        src = os.path.join(CSRC, f)
        obj = os.path.join(BUILD_DIR, f + ".o")
        objs.append(obj)
        cmd = [nvcc, "-std=c++17", "-O3", "-lineinfo", "-Xcompiler", "-fPIC", "-c", src, "-o", obj]
        if f.endswith(".cu"):
            cmd[1:1] = ARCH
        if verbose:
            print(" ".join(cmd))
        jobs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for cmd, p in jobs:
        out, _ = p.communicate()
        if p.returncode != 0:
            failed.append(" ".join(cmd) + "\n" + out.decode(errors="replace"))
    if failed:
        raise RuntimeError("nvcc failed:\n" + "\n".join(failed))
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = [nvcc] + ARCH + ["-shared", "-Xlinker", "--no-undefined", "-o", tmp] + objs
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import time
    t = time.time()
    print(build(force=True, verbose=True), "%.1fs" % (time.time() - t))
