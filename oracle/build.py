"""Compile the FP64 CPU oracle (lbsc_oracle.c, D2Q9, and lbsc3_oracle.c, D3Q19)
into an in-tree shared library.

Test infrastructure only: the oracle is built so that the test suite, the
package smoke check and the benchmark's CPU-baseline leg can load it.  The
product library never links or loads it.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
SRC = os.path.join(HERE, "lbsc_oracle.c")
SRC3 = os.path.join(HERE, "lbsc3_oracle.c")
LIB = os.path.join(HERE, "liblbsc_oracle.so")


def build(force: bool = False) -> str:
    """Build liblbsc_oracle.so next to its source (portable flags: the same
    command builds on x86_64 and aarch64). Returns the library path."""
    if (not force and os.path.exists(LIB)
            and os.path.getmtime(LIB) >= max(os.path.getmtime(SRC), os.path.getmtime(SRC3))):
        return LIB
    tmp = LIB + ".tmp"
    cmd = ["gcc", "-O2", "-fPIC", "-shared", "-std=c11",
           "-fno-fast-math", "-ffp-contract=off", "-fopenmp", "-o", tmp, SRC, SRC3, "-lm",
           "-fopenmp"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
