"""Compile the C oracle (the plain single-threaded form and its row-parallel restatement)
into ``oracle/liboracle.so`` (plain gcc, no architecture flags, no fast-math, no FMA
contraction, so the same IEEE double arithmetic runs on x86-64 and AArch64)."""
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


SOURCES = ("gee_oracle.c", "gee_oracle_rows.c")


def sources():
    return [os.path.join(_HERE, f) for f in SOURCES]


def build_oracle() -> str:
    out = library_path()
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-pthread", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp] + sources() + ["-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle())
