"""Builds the oracle (test infrastructure): liboracle.so from plain C, -ffp-contract=off."""
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))


def build(force: bool = False) -> None:
    srcs = sorted(glob.glob(os.path.join(HERE, "*.c")))
    deps = srcs + sorted(glob.glob(os.path.join(HERE, "*.h")))
    out = os.path.join(HERE, "liboracle.so")
    if force or not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in deps):
        subprocess.check_call(["gcc", "-O2", "-std=gnu11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-pthread", "-Wall", "-Wno-unused-function"] + srcs + ["-o", out, "-lm"])


if __name__ == "__main__":
    build(force=True)
