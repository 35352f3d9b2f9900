"""Build libmarinegym.so in-tree with nvcc for sm_103a (B300).

Usage: python -m paper_2503_09203_b300.build [--force]
"""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
INCLUDE = os.path.join(ROOT, "include")
LIB = os.environ.get("MG_LIB_PATH") or os.path.join(HERE, "libmarinegym.so")
BUILD_DIR = os.path.join(HERE, "_build", os.path.basename(LIB))

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVFLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
           "--expt-relaxed-constexpr"] + os.environ.get("MG_NVCC_EXTRA", "").split()


def _nvcc() -> str:
    for cand in (os.environ.get("NVCC"), shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found")


def sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = sources() + glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return any(os.path.getmtime(p) > t for p in deps)


# Kernel headers the library compiles again at run time (class-specialised
# step kernels, NVRTC); embedded as strings in the library.
JIT_HEADERS = ("mg_rtc.h", "mg_internal.h", "mg_device.cuh", "mg_step.cuh", "mg_adjoint.cuh")


def write_jit_sources(out_dir: str) -> None:
    bodies = []
    for name in JIT_HEADERS:
        text = open(os.path.join(CSRC, name)).read()
        if ")MGJIT" in text:
            raise RuntimeError(f"{name} contains the raw-string delimiter")
        bodies.append(text)
    lines = ["// Generated by build.py: the kernel headers for the run-time compiler.",
             f"static const int kJitHeaderCount = {len(JIT_HEADERS)};",
             "static const char* const kJitHeaderNames[] = {" + ", ".join(f'"{n}"' for n in JIT_HEADERS) + "};",
             "static const char* const kJitHeaderBodies[] = {"]
    lines += [f'R"MGJIT({b})MGJIT",' for b in bodies]
    lines.append("};")
    path = os.path.join(out_dir, "mg_jit_sources.inc")
    new = "\n".join(lines) + "\n"
    if not os.path.exists(path) or open(path).read() != new:
        with open(path, "w") as f:
            f.write(new)


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    write_jit_sources(BUILD_DIR)
    nvcc = _nvcc()
    objs = []
    procs = []
    for src in sources():
        obj = os.path.join(BUILD_DIR, os.path.basename(src) + ".o")
        cmd = [nvcc] + ARCH + NVFLAGS + ["-c", src, "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        else:
            cmd = [nvcc] + NVFLAGS + ["-I", BUILD_DIR, "-x", "c++", "-c", src, "-o", obj]
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
        objs.append(obj)
    failed = False
    for cmd, p in procs:
        out = p.communicate()[0].decode()
        if p.returncode != 0:
            failed = True
            sys.stderr.write(" ".join(cmd) + "\n" + out + "\n")
        elif verbose and out.strip():
            sys.stderr.write(out)
    if failed:
        raise RuntimeError("libmarinegym build failed")
    tmp = LIB + f".tmp{os.getpid()}"
    subprocess.check_call([nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lpthread", "-ldl"])
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
