"""In-tree build of libmmc.so for sm_103a (nvcc, no cmake).

Each translation unit is compiled in parallel to an object under _build/, then
linked into paper_2106_05593_gb300/libmmc.so against the CUDA runtime and cuFFT.
build(checked=True) makes the bounds-checked variant (-DMMC_CHECKED, objects
under _build_checked/) as libmmc_checked.so.
"""
from __future__ import annotations

import concurrent.futures as cf
import os
import shutil
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libmmc.so")
LIB_CHECKED = os.path.join(HERE, "libmmc_checked.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["capi.cu", "k_sweep.cu", "k_demag.cu", "k_demag_il_f16.cu", "k_demag_il_f32.cu", "k_demag_il_f16h.cu",
           "k_demag_il_d16.cu", "k_demag_w32.cu", "k_reduce.cu", "k_grad.cu", "noalloc.cu", "k_serial.cu", "k_sdesc.cu", "k_angles.cu", "k_terms.cu",
           "k_cufft.cu", "host_physics.cpp"]


def _nvcc() -> str:
    for cand in (shutil.which("nvcc"), "/usr/local/cuda/bin/nvcc"):
        if cand and os.path.exists(cand):
            return cand
    raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libmmc.so")


def _stale(obj: str, deps: list[str]) -> bool:
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force: bool = False, verbose: bool = False, extra: list[str] | None = None, checked: bool = False) -> str:
    nvcc = _nvcc()
    bdir = BUILD + "_checked" if checked else BUILD
    lib = LIB_CHECKED if checked else LIB
    extra = (extra or []) + (["-DMMC_CHECKED"] if checked else [])
    os.makedirs(bdir, exist_ok=True)
    headers = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".h", ".cuh"))]
    headers.append(os.path.join(INCLUDE, "mmc.h"))
    flags = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
             "--expt-relaxed-constexpr"] + ARCH + (extra or [])
    jobs = []
    objs = []
    for src in SOURCES:
        path = os.path.join(CSRC, src)
        obj = os.path.join(bdir, src + ".o")
        objs.append(obj)
        if force or _stale(obj, [path] + headers):
            cmd = [nvcc, "-c", path, "-o", obj] + flags
            if src.endswith(".cpp"):
                cmd = [nvcc, "-x", "cu", "-c", path, "-o", obj] + flags
            jobs.append(cmd)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("compile failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for out in ex.map(run, jobs):
                if verbose and out.strip():
                    print(out)
    if force or jobs or not os.path.exists(lib):
        tmp = lib + f".tmp{os.getpid()}"
        cmd = [nvcc, "-shared", "-o", tmp] + objs + ARCH + ["-lcufft", "-lcudart", "-Xcompiler", "-fPIC"]
        run(cmd)
        os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(verbose=True))
