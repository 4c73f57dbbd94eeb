"""Build the CPU oracle (test infrastructure only).

Compiles oracle.c twice with gcc: REAL=double -> _build/liboracle.so and
REAL=long double -> _build/liboracle_ld.so.  ISO C11 with FP contraction off,
so x86-64 and aarch64 hosts evaluate the same expression trees.  The counting
instantiation (count_flops.cpp, oracle.c with REAL = an operation-recording
type) is compiled with g++ into _build/liboracle_count.so.
"""
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
BUILD = os.path.join(HERE, "_build")
VARIANTS = {"liboracle.so": "double", "liboracle_ld.so": "long double"}


def lib_path(name: str) -> str:
    return os.path.join(BUILD, name)


def build(force: bool = False) -> None:
    os.makedirs(BUILD, exist_ok=True)
    src = os.path.join(HERE, "oracle.c")
    hdr = os.path.join(HERE, "oracle.h")
    newest = max(os.path.getmtime(src), os.path.getmtime(hdr))
    procs = []
    for name, real in VARIANTS.items():
        out = lib_path(name)
        if not force and os.path.exists(out) and os.path.getmtime(out) >= newest:
            continue
        cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off",
               f"-DREAL={real}", "-o", out + ".tmp", src, "-lm"]
        procs.append((subprocess.Popen(cmd), out))
    cnt_src = os.path.join(HERE, "count_flops.cpp")
    cnt_out = lib_path("liboracle_count.so")
    cnt_new = max(newest, os.path.getmtime(cnt_src))
    cnt = None
    if force or not os.path.exists(cnt_out) or os.path.getmtime(cnt_out) < cnt_new:
        # C++ reads the C source: -fpermissive lets malloc's void* convert implicitly
        cmd = ["g++", "-std=c++17", "-O1", "-fPIC", "-shared", "-fpermissive", "-w",
               "-ffp-contract=off", "-o", cnt_out + ".tmp", cnt_src, "-lm"]
        try:
            cnt = subprocess.Popen(cmd)
        except OSError:  # no C++ compiler: the counting library (CPU tests only) is skipped
            cnt = None
    for p, out in procs:
        if p.wait() != 0:
            raise RuntimeError(f"oracle build failed for {out}")
        os.replace(out + ".tmp", out)
    if cnt is not None:
        if cnt.wait() == 0:
            os.replace(cnt_out + ".tmp", cnt_out)
        else:
            print("oracle: the counting library did not build (needed by the flop-count test only)",
                  file=sys.stderr)


if __name__ == "__main__":
    build(force="--force" in sys.argv)
    print("oracle built in", BUILD)
