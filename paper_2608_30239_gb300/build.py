"""Build the in-tree shared library `_build/libmcpd.so` for sm_103a (GB300).

Translation units compiled in parallel: the host table builder (g++, -ffp-contract=off so every
double expression keeps its written order), the C ABI (g++), and the kernels (nvcc,
`-gencode arch=compute_103a,code=sm_103a`: the sampling kernel's single-instance variants, its
batched variants, its trajectory-recording variants, the no-allocation entry point, the learned model, the lane-group
kernel).  No cmake; a rebuild happens only when a source is
newer than the library.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libmcpd.so")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
ARCH = "-gencode=arch=compute_103a,code=sm_103a"


def _cuda_home() -> str:
    for cand in (os.environ.get("CUDA_HOME"), "/usr/local/cuda"):
        if cand and os.path.exists(os.path.join(cand, "bin", "nvcc")):
            return cand
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(nvcc))
    raise RuntimeError("nvcc not found: set CUDA_HOME")


def sources():
    return [os.path.join(SRC, f) for f in ("mcpd_tables.cpp", "mcpd_api.cpp", "mcpd_kernels.cu",
                                           "mcpd_trace.cu", "mcpd_batch.cu", "mcpd_batch_deg.cu", "mcpd_batch_ext.cu",
                                           "mcpd_noalloc.cu", "mcpd_mlp.cu", "mcpd_group.cu",
                                           "mcpd_internal.h", "mcpd_device.cuh", "mcpd_pairs.cuh")] + \
        [os.path.join(INCLUDE, "mcpd.h")]


def needs_build() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(s) > t for s in sources() if os.path.exists(s))


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False) -> str:
    if not force and not needs_build():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cuda = _cuda_home()
    nvcc = os.path.join(cuda, "bin", "nvcc")
    inc = ["-I" + INCLUDE, "-I" + SRC, "-I" + os.path.join(cuda, "include")]
    objs = {name: os.path.join(BUILD, name + ".o")
            for name in ("tables", "api", "kernels", "trace", "batch", "batch_deg", "batch_ext", "noalloc", "mlp",
                         "group")}
    cxx = ["g++", "-O2", "-std=c++17", "-fPIC", "-ffp-contract=off", "-fno-fast-math", "-Wall"]
    jobs = [
        cxx + inc + ["-c", os.path.join(SRC, "mcpd_tables.cpp"), "-o", objs["tables"]],
        cxx + inc + ["-c", os.path.join(SRC, "mcpd_api.cpp"), "-o", objs["api"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]
        + (["-Xptxas", "-v"] if ptxas_info else []) + inc
        + ["-c", os.path.join(SRC, "mcpd_kernels.cu"), "-o", objs["kernels"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]
        + inc + ["-c", os.path.join(SRC, "mcpd_trace.cu"), "-o", objs["trace"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]
        + inc + ["-c", os.path.join(SRC, "mcpd_batch.cu"), "-o", objs["batch"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]
        + inc + ["-c", os.path.join(SRC, "mcpd_batch_deg.cu"), "-o", objs["batch_deg"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]
        + inc + ["-c", os.path.join(SRC, "mcpd_batch_ext.cu"), "-o", objs["batch_ext"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off"]
        + inc + ["-c", os.path.join(SRC, "mcpd_noalloc.cu"), "-o", objs["noalloc"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
        + inc + ["-c", os.path.join(SRC, "mcpd_mlp.cu"), "-o", objs["mlp"]],
        [nvcc, ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC"]
        + (["-Xptxas", "-v"] if ptxas_info else []) + inc
        + ["-c", os.path.join(SRC, "mcpd_group.cu"), "-o", objs["group"]],
    ]
    procs = [subprocess.Popen(j, stdout=subprocess.PIPE, stderr=subprocess.STDOUT) for j in jobs]
    logs = []
    for j, p in zip(jobs, procs):
        out, _ = p.communicate()
        logs.append(out.decode(errors="replace"))
        if p.returncode != 0:
            raise RuntimeError("build failed: " + " ".join(j) + "\n" + logs[-1])
    if verbose or ptxas_info:
        sys.stdout.write("".join(logs))
    tmp = LIB + f".tmp{os.getpid()}"
    link = [nvcc, ARCH, "-shared", "-o", tmp, objs["tables"], objs["api"], objs["kernels"], objs["trace"],
            objs["batch"], objs["batch_deg"], objs["batch_ext"], objs["noalloc"], objs["mlp"], objs["group"],
            "-cudart", "static"]
    subprocess.check_call(link)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
