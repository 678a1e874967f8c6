"""Build the CUDA library in-tree: every csrc/*.cu compiled for sm_103a in parallel, then linked into
paper_2305_01537_gb300/libsph_filter.so. Run `python -m paper_2305_01537_gb300.build`."""
from __future__ import annotations

import glob
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OBJ = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libsph_filter.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                     "-Xcompiler", "-ffp-contract=off", "-Xptxas", "-warn-spills"]


def nvcc() -> str:
    path = shutil.which("nvcc")
    if path:
        return path
    cand = "/usr/local/cuda/bin/nvcc"
    if os.path.exists(cand):
        return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")


# shell_inst.cu is compiled once per (precision, FFT length, hybrid variant) instantiation of the
# shell kernels (for length 256 the hybrid object holds only the cluster-pair kernel)
SHELL_INST = [(d, n, h) for d in (0, 1) for n in (0, 32, 64, 96, 128, 192, 256) for h in (0, 1)]
SHELL_INST += [(2, 0, 0), (2, 128, 0)]  # the FP64 spectral form


def jobs():
    """(source, object, extra flags) for every compilation."""
    out = []
    for src in sorted(glob.glob(os.path.join(CSRC, "*.cu"))):
        base = os.path.basename(src)[:-3]
        if base == "shell_inst":
            for d, n, h in SHELL_INST:
                out.append((src, os.path.join(OBJ, f"shell_inst_d{d}_n{n}_h{h}.o"),
                            [f"-DSPH_SHELL_DF={d}", f"-DSPH_SHELL_LEN={n}", f"-DSPH_SHELL_HYB={h}"]))
        else:
            out.append((src, os.path.join(OBJ, base + ".o"), []))
    return out


def _stale(obj: str, deps) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(OBJ, exist_ok=True)
    headers = (glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh"))
               + glob.glob(os.path.join(HERE, "..", "include", "*.h")))
    objs, procs = [], []
    for src, obj, extra in jobs():
        objs.append(obj)
        if force or _stale(obj, [src] + headers):
            cmd = [nvcc()] + NVCC_FLAGS + extra + ["-c", src, "-o", obj]
            if verbose:
                print(" ".join(cmd))
            procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    failed = []
    for src, p in procs:
        out, _ = p.communicate()
        text = out.decode(errors="replace")
        if p.returncode != 0:
            failed.append((src, text))
        elif verbose and text.strip():
            print(text)
    if failed:
        msg = "\n".join(f"--- {s}\n{t}" for s, t in failed)
        raise RuntimeError(f"nvcc failed:\n{msg}")
    if force or procs or not os.path.exists(LIB) or _stale(LIB, objs):
        cmd = [nvcc()] + ARCH + ["-shared", "-o", LIB + ".tmp"] + objs + ["-lcudart"]
        subprocess.run(cmd, check=True)
        os.replace(LIB + ".tmp", LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True)
    print(LIB)
