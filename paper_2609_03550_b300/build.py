"""Build the CUDA library (libqds.so, sm_103a) and the host emulator of its
step kernels (libqds_emu.so, CPU tests only) in the package directory."""
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libqds.so")
EMU = os.path.join(HERE, "libqds_emu.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["qds_api.cu", "qds_noalloc.cu", "qds_adjoint.cu", "qds_modes.cu", "qds_inputs.cu"]
HEADERS = ["qds_common.cuh", "qds_stages.cuh", "qds_kernels.cuh", "qds_march.cuh", "qds_adjoint.cuh"]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build_cuda(force=False, verbose=False):
    deps = [os.path.join(CSRC, f) for f in SOURCES + HEADERS] + [os.path.join(HERE, "..", "include", "qds.h")]
    if not force and not _stale(LIB, deps):
        return LIB
    cmd = [NVCC, *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-o", LIB + ".tmp", *[os.path.join(CSRC, f) for f in SOURCES]]
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    subprocess.check_call(cmd)
    os.replace(LIB + ".tmp", LIB)
    return LIB


def build_emu(force=False):
    deps = [os.path.join(CSRC, f) for f in ("qds_emu.cpp", "qds_common.cuh", "qds_stages.cuh", "qds_march.cuh",
                                            "qds_adjoint.cuh")]
    if not force and not _stale(EMU, deps):
        return EMU
    cmd = ["g++", "-O2", "-std=c++17", "-fPIC", "-shared", "-Wno-unknown-pragmas",
           "-o", EMU + ".tmp", os.path.join(CSRC, "qds_emu.cpp")]
    subprocess.check_call(cmd)
    os.replace(EMU + ".tmp", EMU)
    return EMU


def build(force=False):
    build_emu(force)
    return build_cuda(force)


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv))
