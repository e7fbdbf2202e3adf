"""The library's host code under AddressSanitizer and UndefinedBehaviorSanitizer (no GPU needed).

Builds mcpd_tables.cpp and mcpd_api.cpp with both sanitizers, with stand-ins for the kernel
launchers (stubs.cpp), loads that build in place of the library, and runs the host tests of
tests/test_abi.py (all but the export check, which the stand-ins cannot pass) with the sanitized
oracle beside it.  Any report aborts the run.

  python tests/sanitize_host/run.py
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
sys.path.insert(0, ROOT)

from paper_2608_30239_gb300 import build as lib_build  # noqa: E402


def runtime(name):
    return subprocess.check_output(["gcc", f"-print-file-name={name}"], text=True).strip()


def build_host_library():
    out_dir = os.path.join(HERE, "_build")
    os.makedirs(out_dir, exist_ok=True)
    lib = os.path.join(out_dir, "libmcpd_host_san.so")
    cuda = lib_build._cuda_home()
    src = lib_build.SRC
    subprocess.check_call(
        ["g++", "-std=c++17", "-O1", "-g", "-fPIC", "-shared", "-fno-omit-frame-pointer",
         "-fsanitize=address,undefined", "-fno-sanitize-recover=undefined", "-ffp-contract=off",
         "-I" + lib_build.INCLUDE, "-I" + src, "-I" + os.path.join(cuda, "include"),
         os.path.join(src, "mcpd_api.cpp"), os.path.join(src, "mcpd_tables.cpp"),
         os.path.join(HERE, "stubs.cpp"), "-o", lib,
         "-L" + os.path.join(cuda, "lib64"), "-lcudart", "-Wl,-rpath," + os.path.join(cuda, "lib64")])
    return lib


def main():
    if "libasan" not in os.environ.get("LD_PRELOAD", ""):
        lib = build_host_library()
        env = dict(os.environ, LD_PRELOAD=f"{runtime('libasan.so')}:{runtime('libubsan.so')}",
                   ASAN_OPTIONS="detect_leaks=0", MCPD_ORACLE_SANITIZE="1", MCPD_HOST_SAN_LIB=lib)
        os.execve(sys.executable, [sys.executable, os.path.abspath(__file__)] + sys.argv[1:], env)
    lib_build.LIB = os.environ["MCPD_HOST_SAN_LIB"]
    lib_build.build = lambda *a, **k: lib_build.LIB
    import pytest
    return pytest.main(["-q", "-p", "no:cacheprovider", "-m", "not gpu",
                        os.path.join(ROOT, "tests", "test_abi.py"), "-k", "not exports_every_declared"]
                       + sys.argv[1:])


if __name__ == "__main__":
    sys.exit(main())
