"""Build the in-tree CUDA library libmsclbm.so for sm_103a with nvcc.

Run as ``python -m paper_2609_39474_b300.build`` (or through ``__graft_entry__.build()``).
The shared object is written next to this file so that it travels with the source tree.
"""
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
LIB = os.path.join(HERE, "libmsclbm.so")
# bounds-checked debug build: every MSC_INB index check compiled in (msc_bounds_check_report)
LIB_CHECK = os.path.join(HERE, "libmsclbm_check.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc_path() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmsclbm.so")


def sources():
    return [os.path.join(CSRC, f) for f in sorted(os.listdir(CSRC)) if f.endswith((".cu", ".cuh"))]


def up_to_date(lib: str) -> bool:
    if not os.path.exists(lib):
        return False
    t = os.path.getmtime(lib)
    hdr = os.path.join(os.path.dirname(HERE), "include", "msclbm.h")
    return all(os.path.getmtime(s) <= t for s in sources() + [hdr, __file__])


def build(force: bool = False, verbose: bool = False, variant: str = "") -> str:
    """Compile libmsclbm.so (variant "") or the bounds-checked libmsclbm_check.so (variant "check")."""
    if variant not in ("", "check"):
        raise ValueError(f"unknown variant {variant!r}")
    lib = LIB_CHECK if variant == "check" else LIB
    if not force and up_to_date(lib):
        return lib
    cmd = [nvcc_path(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-shared",
           "-o", lib + ".tmp", os.path.join(CSRC, "msclbm.cu")]
    if variant == "check":
        cmd.insert(1, "-DMSC_BOUNDS_CHECK")
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError("nvcc failed:\n" + res.stdout + res.stderr)
    if verbose:
        sys.stderr.write(res.stderr)
    os.replace(lib + ".tmp", lib)
    return lib


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv,
                variant="check" if "--check" in sys.argv else ""))
