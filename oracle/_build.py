"""Compile the C oracle into ``oracle/liboracle.so`` (plain gcc, no architecture flags,
no fast-math, so the same IEEE double arithmetic runs on x86-64 and AArch64)."""
import os
import subprocess

_HERE = os.path.dirname(os.path.abspath(__file__))


def library_path() -> str:
    return os.path.join(_HERE, "liboracle.so")


def build_oracle() -> str:
    out = library_path()
    tmp = out + f".tmp{os.getpid()}"
    cmd = ["gcc", "-O2", "-std=c11", "-fPIC", "-shared", "-fno-fast-math", "-ffp-contract=off",
           "-o", tmp, os.path.join(_HERE, "gee_oracle.c"), "-lm"]
    subprocess.run(cmd, check=True)
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build_oracle())
