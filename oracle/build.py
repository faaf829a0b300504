"""Build the oracle shared library (test infrastructure only).

Compiles the plain C++17 sources of this directory into ``liboracle.so`` next
to them. Portable host code only (x86-64 and aarch64): no intrinsics, no
``-march=native``.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
SOURCES = ["orc_rng.cpp", "orc_hbitmap.cpp", "orc_gol.cpp", "orc_wator.cpp", "orc_nbody.cpp", "orc_traffic.cpp", "orc_sugarscape.cpp"]
LIB = os.path.join(HERE, "liboracle.so")


def build(force: bool = False) -> str:
    srcs = [os.path.join(HERE, s) for s in SOURCES] + [os.path.join(HERE, "oracle.h")]
    if not force and os.path.exists(LIB):
        lib_m = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= lib_m for s in srcs):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["g++", "-std=c++17", "-O2", "-fPIC", "-shared", "-pthread", "-o", tmp] + [os.path.join(HERE, s) for s in SOURCES]
    subprocess.check_call(cmd)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv))
