"""Build the CUDA library librti.so in-tree (nvcc, sm_103a only).

Three translation units compile in parallel: the binary64 kernels (-fmad=false, so
every product and sum rounds separately), the binary32 kernels, and the host side
of the C ABI. The result lands in paper_2408_07609_gb300/_build/.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(BUILD, "librti.so")
LIB_CHECKED = os.path.join(BUILD, "librti_checked.so")
NVCC = os.environ.get("NVCC", "/usr/local/cuda/bin/nvcc")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", os.path.join(ROOT, "include"),
          "-I", CSRC, "-Xcompiler", "-ffp-contract=off"]
UNITS = {
    "rti_fp64.cu": ["-fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "rti_fp32.cu": [],
    "rti_host.cu": ["-Xcompiler", "-pthread"],
}


def _sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC))]


def _stale(lib=LIB):
    if not os.path.exists(lib):
        return True
    t = os.path.getmtime(lib)
    deps = _sources() + [os.path.join(ROOT, "include", "rti.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def build(force: bool = False, verbose: bool = False, ptxas_info: bool = False,
          checked: bool = False) -> str:
    """checked=True builds librti_checked.so with every kernel index range-checked."""
    out = LIB_CHECKED if checked else LIB
    if not force and not _stale(out):
        return out
    os.makedirs(BUILD, exist_ok=True)
    objs = []

    def one(unit):
        src = os.path.join(CSRC, unit)
        obj = os.path.join(BUILD, unit.replace(".cu", "_chk.o" if checked else ".o"))
        cmd = [NVCC, *ARCH, *COMMON, *UNITS[unit], "-c", src, "-o", obj]
        if checked:
            cmd.append("-DRTI_CHECKED")
        if ptxas_info:
            cmd += ["-Xptxas", "-v"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {unit}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(UNITS)) as ex:
        for obj, log in ex.map(one, list(UNITS)):
            objs.append(obj)
            if verbose and log:
                sys.stderr.write(log)
    tmp = out + f".tmp{os.getpid()}"
    r = subprocess.run([NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static",
                        "-Xcompiler", "-pthread"],
                       capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, out)
    return out


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_info="--ptxas" in sys.argv))
