"""Builds the input generator: libsynth_host.so (gcc) and libsynth_dev.so (nvcc, sm_103a)."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")


def _stale(out, srcs):
    return not os.path.exists(out) or any(os.path.getmtime(s) > os.path.getmtime(out) for s in srcs)


def build(force: bool = False) -> None:
    hdr = os.path.join(HERE, "synth_common.h")
    host_src = os.path.join(HERE, "synth_host.c")
    host_out = os.path.join(HERE, "libsynth_host.so")
    if force or _stale(host_out, [host_src, hdr]):
        subprocess.check_call(["gcc", "-O2", "-std=c11", "-ffp-contract=off", "-fno-fast-math", "-fPIC", "-shared",
                               "-pthread", host_src, "-o", host_out, "-lm"])
    dev_src = os.path.join(HERE, "synth_dev.cu")
    dev_out = os.path.join(HERE, "libsynth_dev.so")
    if force or _stale(dev_out, [dev_src, hdr]):
        subprocess.check_call([NVCC, "-O3", "-std=c++17", "-gencode", "arch=compute_103a,code=sm_103a", "-lineinfo",
                               "-Xcompiler", "-fPIC", "-shared", dev_src, "-o", dev_out])


if __name__ == "__main__":
    build(force=True)
