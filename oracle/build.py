"""Compile the C part of the oracle (``fz_oracle.c``) into ``liboracle.so``.

TEST INFRASTRUCTURE: building the checker is not using it.  ``build()`` in
``__graft_entry__`` calls :func:`build_oracle`; the oracle loader calls it too
when the shared object is missing or older than its source.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "fz_oracle.c")
LIB = os.path.join(HERE, "liboracle.so")


def build_oracle(force: bool = False) -> str:
    """Build ``liboracle.so`` with gcc (plain C99, portable flags) and return its path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= os.path.getmtime(SRC)):
        return LIB
    tmp = LIB + ".tmp.%d" % os.getpid()
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread",
           "-Wall", "-Wextra", "-o", tmp, SRC]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build_oracle(force=True))
