"""Build of the in-tree CUDA library ``_build/libft.so`` for sm_103a.

The kernel instantiations are split into several translation units (one per
padded rank K and precision) that nvcc compiles in parallel; the host C ABI
is one more unit.  The result is linked with the static CUDA runtime, so the
library depends only on the driver.
"""
from __future__ import annotations

import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
OUT_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(OUT_DIR, "libft.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2",
              f"-I{INCLUDE}", f"-I{CSRC}"]

# (source, extra defines, object name)
UNITS = [("ft_api.cu", [], "ft_api"), ("ft_batch.cu", [], "ft_batch"), ("ft_stepnet.cu", [], "ft_stepnet")]
# the slowest units first, so a parallel build finishes early
for _m in (0, 1, 2):
    for _k in (32, 16):
        for _n in range(5 if _k == 32 else 10, 0, -1):
            UNITS.append(("ft_inst.cu", [f"-DFT_K={_k}", f"-DFT_MATH={_m}", f"-DFT_N={_n}"],
                          f"ft_inst_{_k}_{_m}_{_n}"))
for _k in (16, 32):
    UNITS.append(("ft_eval.cu", [f"-DFT_K={_k}"], f"ft_eval_{_k}"))


def nvcc() -> str:
    cand = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build the library")
    return cand


def _sources_digest(extra=(), csrc=CSRC) -> str:
    h = hashlib.sha256()
    for name in sorted(os.listdir(csrc)):
        with open(os.path.join(csrc, name), "rb") as f:
            h.update(name.encode())
            h.update(f.read())
    with open(os.path.join(INCLUDE, "ft.h"), "rb") as f:
        h.update(f.read())
    h.update(" ".join(ARCH + NVCC_FLAGS + list(extra)).encode())
    return h.hexdigest()


def build(force: bool = False, jobs: int | None = None, verbose: bool = False,
          extra_defines=(), out_dir: str | None = None, csrc: str = CSRC) -> str:
    """Compile every unit (in parallel) and link ``libft.so``; skipped when the
    sources are unchanged since the last build.  ``extra_defines`` and
    ``out_dir`` build a variant elsewhere (e.g. another cache policy);
    ``csrc`` compiles another source tree with the same flags."""
    out_dir = out_dir or OUT_DIR
    lib_path = os.path.join(out_dir, "libft.so")
    os.makedirs(out_dir, exist_ok=True)
    stamp = os.path.join(out_dir, "sources.sha256")
    digest = _sources_digest(extra_defines, csrc)
    if not force and os.path.exists(lib_path) and os.path.exists(stamp):
        with open(stamp) as f:
            if f.read().strip() == digest:
                return lib_path
    exe = nvcc()
    jobs = jobs or max(1, min(len(UNITS), len(os.sched_getaffinity(0)) if hasattr(os, "sched_getaffinity")
                                 else (os.cpu_count() or 1)))

    def compile_unit(unit):
        src, defs, name = unit
        obj = os.path.join(out_dir, name + ".o")
        flags = [f if f != f"-I{CSRC}" else f"-I{csrc}" for f in NVCC_FLAGS]
        cmd = [exe, *ARCH, *flags, *extra_defines, *defs, "-c", os.path.join(csrc, src), "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {name}:\n{r.stderr}")
        if verbose and r.stderr:
            print(r.stderr)
        return obj

    with cf.ThreadPoolExecutor(max_workers=jobs) as pool:
        objs = list(pool.map(compile_unit, UNITS))
    tmp = lib_path + f".tmp{os.getpid()}"
    cmd = [exe, *ARCH, "-shared", "-cudart", "static", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, lib_path)
    with open(stamp, "w") as f:
        f.write(digest)
    return lib_path


if __name__ == "__main__":  # pragma: no cover
    import time
    t = time.time()
    print(build(force=True, verbose=False), f"{time.time() - t:.1f}s")
