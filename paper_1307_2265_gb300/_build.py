"""Build of libenzo_ppm.so for sm_103a with nvcc (in-tree, no cmake).

Translation units and their flags:
  abi.cu        host entry points, work lists, ghost fill, CFL finalisation
  fp64_path.cu  FP64 sweep/CFL/Riemann: --fmad=false, IEEE div and sqrt
  fp32_path.cu  FP32 sweep/CFL/Riemann: -use_fast_math (FMA, fast rcp/sqrt)
  noalloc.cu    sweep entry point whose scratch is a library-owned device array
  hierarchy.cu  ghost fill from parents/siblings, flux correction, projection (FP64,
                --fmad=false)
  mlp.cu        learned p* guess: tcgen05 inference and training kernels
  amr.cu        hierarchy rebuild: cell flagging (FP64, --fmad=false) and the
                host clustering of flags into new grids
  probe.cu      FP64-pipe throughput probe (the FP64 sweep's roofline denominator)
  driver.cu     AMR hierarchy driver: level plans, the EvolveLevel W-cycle, rebuilds
                (host code calling the entry points above)
Objects go to paper_1307_2265_gb300/_build/, the library next to this file.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(PKG, "_build")
LIB = os.path.join(PKG, "libenzo_ppm.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
COMMON = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC]
UNITS = {
    "abi.cu": [],
    "fp64_path.cu": ["--fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "fp32_path.cu": ["-use_fast_math"],
    "noalloc.cu": [],
    "mlp.cu": ["-use_fast_math"],
    "hierarchy.cu": ["--fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "amr.cu": ["--fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "probe.cu": ["--fmad=false", "-prec-div=true", "-prec-sqrt=true"],
    "driver.cu": [],
}
OPTIONAL_UNITS = {}


def nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libenzo_ppm")


def _units():
    u = dict(UNITS)
    for name, flags in OPTIONAL_UNITS.items():
        if os.path.exists(os.path.join(CSRC, name)):
            u[name] = flags
    return u


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    srcs = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    srcs.append(os.path.abspath(__file__))
    return any(os.path.getmtime(s) > t for s in srcs)


def build(force: bool = False, verbose: bool = False, extra=()) -> str:
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    cc = nvcc()
    units = _units()

    def compile_one(name):
        obj = os.path.join(BUILD, name.replace(".cu", ".o"))
        cmd = [cc, *ARCH, *COMMON, *units[name], *extra, "-c", os.path.join(CSRC, name), "-o", obj]
        if verbose:
            print(" ".join(cmd))
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stdout}\n{r.stderr}")
        return obj, r.stderr

    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        results = list(ex.map(compile_one, sorted(units)))
    if verbose:
        for _, err in results:
            if err.strip():
                print(err)
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [cc, *ARCH, "-shared", "-o", tmp] + [o for o, _ in results] + ["-lcudart"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose=True, extra=sys.argv[1:]))
