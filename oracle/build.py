"""Build the oracle's C library (test infrastructure only).

Compiles ``oracle/newell.c`` with gcc into ``oracle/_build/liboracle_newell.so``.
Only the tests, ``__graft_entry__.smoke()`` and ``bench.py``'s CPU-baseline leg
load the result; the CUDA library never links or calls it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
LIB = os.path.join(HERE, "_build", "liboracle_newell.so")
SOURCES = [os.path.join(HERE, "newell.c"), os.path.join(HERE, "newell_impl.h")]


def build(force: bool = False) -> str:
    """Compile the oracle library if it is missing or older than its sources."""
    os.makedirs(os.path.dirname(LIB), exist_ok=True)
    if not force and os.path.exists(LIB):
        lib_mtime = os.path.getmtime(LIB)
        if all(os.path.getmtime(s) <= lib_mtime for s in SOURCES):
            return LIB
    tmp = LIB + ".tmp%d" % os.getpid()
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-fopenmp", "-Wall", "-o", tmp,
           os.path.join(HERE, "newell.c"), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
