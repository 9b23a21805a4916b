"""Build the CPU oracle (TEST INFRASTRUCTURE) into oracle/_build/libctd_oracle.so.

The oracle is plain C11 compiled with -ffp-contract=off so that the binary32
method takes every multiply and add as a separate IEEE operation on x86_64 and
on aarch64 alike.
"""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libctd_oracle.so")
SOURCES = ["ctd_oracle.c"]
DEPS = SOURCES + ["ctd_oracle.h", "ctd_oracle_transport.inc"]


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    return any(os.path.getmtime(os.path.join(HERE, d)) > t for d in DEPS)


def build(force: bool = False) -> str:
    """Compile the oracle if its sources changed; return the library path."""
    if not force and not _stale():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = ["gcc", "-std=c11", "-O2", "-fPIC", "-shared", "-ffp-contract=off", "-fno-fast-math",
           "-Wall", "-Wno-unused-function", "-o", tmp]
    cmd += [os.path.join(HERE, s) for s in SOURCES] + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True))
