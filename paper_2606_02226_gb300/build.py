"""Builds ``libcfs.so`` in-tree (``paper_2606_02226_gb300/_build/``).

Steps: embed the device sources handed to NVRTC at run time
(``cfs_args.h``, ``cfs_device.cuh``, ``cfs_kernels.cuh``) as C++ raw string
literals; compile every translation unit with nvcc for sm_103a in parallel;
link one shared library against the CUDA runtime and NVRTC.
"""
from __future__ import annotations

import os
import shutil
import subprocess
import sys
import threading
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libcfs.so")

GENCODE = "arch=compute_103a,code=sm_103a"
EMBEDDED = [("kSrcArgs", "cfs_args.h"), ("kSrcDevice", "cfs_device.cuh"),
            ("kSrcKernels", "cfs_kernels.cuh")]
SOURCES = ["cfs_api.cpp", "cfs_batch.cpp", "cfs_codegen.cpp", "cfs_runtime.cpp",
           "cfs_builtin.cu", "cfs_sort.cu", "cfs_sampler.cu", "cfs_noalloc.cu", "cfs_display.cu", "cfs_scribble.cpp",
           "cfs_embed.cpp"]
_LOCK = threading.Lock()


def cuda_home() -> str:
    h = os.environ.get("CUDA_HOME") or os.environ.get("CUDA_PATH")
    if h and os.path.isdir(h):
        return h
    nvcc = shutil.which("nvcc")
    if nvcc:
        return os.path.dirname(os.path.dirname(os.path.realpath(nvcc)))
    return "/usr/local/cuda"


def _write_if_changed(path: str, text: str) -> None:
    if os.path.exists(path):
        with open(path) as fh:
            if fh.read() == text:
                return
    with open(path, "w") as fh:
        fh.write(text)


def _embed() -> str:
    out = ["// generated by build.py: device sources handed to NVRTC", "namespace cfs {"]
    for sym, name in EMBEDDED:
        with open(os.path.join(CSRC, name)) as fh:
            text = fh.read()
        assert ")CFSRAW\"" not in text
        out.append(f'extern const char* const {sym};')
        out.append(f'const char* const {sym} = R"CFSRAW({text})CFSRAW";')
    out.append("}  // namespace cfs")
    path = os.path.join(BUILD, "cfs_embed.cpp")
    _write_if_changed(path, "\n".join(out) + "\n")
    return path


def _inputs_newest() -> float:
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    files.append(os.path.abspath(__file__))
    return max(os.path.getmtime(f) for f in files)


def build(force: bool = False, verbose: bool = False) -> str:
    """Compiles libcfs.so if any source is newer; returns its path."""
    with _LOCK:
        os.makedirs(BUILD, exist_ok=True)
        if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _inputs_newest():
            return LIB
        cuda = cuda_home()
        nvcc = os.path.join(cuda, "bin", "nvcc")
        embed = _embed()
        common = ["-gencode", GENCODE, "-O3", "-lineinfo", "--fmad=false", "-std=c++17",
                  "-Xcompiler", "-fPIC,-O2", "-I", INCLUDE, "-I", CSRC]

        def compile_one(src: str) -> str:
            path = embed if src == "cfs_embed.cpp" else os.path.join(CSRC, src)
            obj = os.path.join(BUILD, os.path.splitext(src)[0] + ".o")
            cmd = [nvcc] + common + ["-c", path, "-o", obj]
            r = subprocess.run(cmd, capture_output=True, text=True)
            if r.returncode != 0:
                raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
            if verbose and (r.stdout or r.stderr):
                sys.stderr.write(r.stdout + r.stderr)
            return obj

        with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
            objs = list(ex.map(compile_one, SOURCES))
        lib64 = os.path.join(cuda, "lib64")
        tmp = LIB + f".{os.getpid()}.tmp"
        cmd = [nvcc, "-shared", "-gencode", GENCODE, "-o", tmp] + objs + [
            "-cudart", "shared", "-L", lib64, "-lnvrtc", "-Xlinker", f"-rpath,{lib64}"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, LIB)
        return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
