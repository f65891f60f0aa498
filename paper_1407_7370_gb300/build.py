"""Build the CUDA library in-tree: paper_1407_7370_gb300/_build/libdirac_gb300.so (sm_103a)."""
from __future__ import annotations

import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
SOURCES = [os.path.join(HERE, "csrc", n) for n in ("dirac_capi.cu", "dirac_step.cu", "dirac_step32.cu",
                                                    "dirac_eigs.cu", "dirac_adjoint.cu")]
DEPS = SOURCES + [os.path.join(HERE, "csrc", "dirac_kernels.cuh"),
                  os.path.join(HERE, "csrc", "dirac_internal.h"),
                  os.path.join(ROOT, "include", "dirac.h")]
OUT_DIR = os.path.join(HERE, "_build")
LIB = os.path.join(OUT_DIR, "libdirac_gb300.so")
ARCH = "arch=compute_103a,code=sm_103a"


def nvcc_path() -> str:
    found = shutil.which("nvcc")
    if found:
        return found
    for cand in ("/usr/local/cuda/bin/nvcc",):
        if os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


def up_to_date() -> bool:
    if not os.path.exists(LIB):
        return False
    t = os.path.getmtime(LIB)
    return all(os.path.getmtime(d) <= t for d in DEPS)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compile the library for sm_103a (cross-compiles without a GPU)."""
    if not force and up_to_date():
        return LIB
    os.makedirs(OUT_DIR, exist_ok=True)
    tag = ".tmp%d" % os.getpid()
    nvcc = nvcc_path()
    flags = ["-std=c++17", "-O3", "-lineinfo", "-gencode", ARCH, "-Xcompiler", "-fPIC",
             "-I", os.path.join(ROOT, "include")]
    # one object per translation unit, compiled in parallel, then one link
    objs, procs = [], []
    for src in SOURCES:
        obj = os.path.join(OUT_DIR, os.path.basename(src) + tag + ".o")
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        objs.append(obj)
        procs.append((cmd, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT,
                                            text=True)))
    out, bad = [], None
    for cmd, p in procs:
        text, _ = p.communicate()
        out.append(text)
        if p.returncode != 0 and bad is None:
            bad = "nvcc failed:\n" + " ".join(cmd) + "\n" + text
    if bad is not None:
        for o in objs:
            if os.path.exists(o):
                os.remove(o)
        raise RuntimeError(bad)
    tmp = LIB + tag
    cmd = [nvcc, "-shared", "-gencode", ARCH, "-o", tmp] + objs
    res = subprocess.run(cmd, capture_output=True, text=True)
    for o in objs:
        os.remove(o)
    if res.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + " ".join(cmd) + "\n" + res.stdout + res.stderr)
    if verbose:
        print("".join(out) + res.stdout + res.stderr)
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force=True, verbose=True))
