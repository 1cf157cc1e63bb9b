"""Builds the native library libps.so in-tree with nvcc for sm_103a.

The translation units (the phase-space kernels, the host compiler/runtime, the coupling
flow, the unweighting, the inverse maps and the FP64-pipe probes) are compiled in parallel and linked into one shared library with the
CUDA runtime linked statically.
"""
from __future__ import annotations

import os
import subprocess
import sys
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
INCLUDE = os.path.join(ROOT, "include")
LIB = os.path.join(HERE, "libps.so")
BUILD_DIR = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["kernels.cu", "graph.cpp", "flow.cu", "unweight.cu", "inverse.cu", "jit.cpp", "probe.cu"]
# device headers that compiled programs (jit.cpp) hand to NVRTC, embedded as text
JIT_HEADERS = [("map_device.cuh", CSRC), ("kin.cuh", CSRC), ("philox.cuh", CSRC), ("launch_params.h", CSRC),
               ("tan_table.h", CSRC), ("ps.h", INCLUDE)]


def nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.sep not in cand or os.path.exists(cand)):
            return cand
    return "nvcc"


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)] + [os.path.join(INCLUDE, "ps.h"), __file__]
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def cuda_lib_dir():
    """lib64 of the toolkit whose nvcc builds the library (libnvrtc is found there at run time)."""
    path = nvcc()
    if os.path.sep not in path:
        from shutil import which
        path = which(path) or path
    return os.path.join(os.path.dirname(os.path.dirname(os.path.realpath(path))), "lib64")


def write_jit_sources(path):
    """The device headers as C++ raw strings (kJitHeaderNames/Texts/Count) for jit.cpp."""
    out = []
    names = []
    for k, (name, d) in enumerate(JIT_HEADERS):
        text = open(os.path.join(d, name)).read()
        assert ")PSJIT" not in text
        out.append(f'const char* const kJitHeader{k} = R"PSJIT({text})PSJIT";')
        names.append(f'"{name}"')
    out.append("const char* const kJitHeaderNames[] = {" + ", ".join(names) + "};")
    out.append("const char* const kJitHeaderTexts[] = {" +
               ", ".join(f"kJitHeader{k}" for k in range(len(JIT_HEADERS))) + "};")
    out.append(f"const int kJitHeaderCount = {len(JIT_HEADERS)};")
    tmp = path + ".tmp"
    with open(tmp, "w") as f:
        f.write("\n".join(out) + "\n")
    os.replace(tmp, path)


def build(force=False, verbose=False, ptxas_verbose=False):
    """Compile the library if any source is newer than libps.so; returns its path."""
    if not force and not _stale():
        return LIB
    os.makedirs(BUILD_DIR, exist_ok=True)
    write_jit_sources(os.path.join(BUILD_DIR, "jit_sources.inc"))
    common = [nvcc(), *ARCH, "-lineinfo", "-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-I", INCLUDE, "-I", CSRC,
              "-I", BUILD_DIR]
    if ptxas_verbose:
        common += ["-Xptxas", "-v"]

    def compile_one(src):
        obj = os.path.join(BUILD_DIR, src + ".o")
        cmd = common + ["-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cpp"):
            cmd = common + ["-x", "cu", "-c", os.path.join(CSRC, src), "-o", obj]
        res = subprocess.run(cmd, capture_output=True, text=True)
        if res.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{res.stdout}\n{res.stderr}")
        if verbose or ptxas_verbose:
            sys.stderr.write(res.stdout + res.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        objs = list(ex.map(compile_one, SOURCES))
    tmp = LIB + ".tmp"
    libdir = cuda_lib_dir()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs, "-cudart", "static", "-L", libdir, "-lnvrtc", "-lnvJitLink", "-ldl",
           "-Xlinker", "-rpath", "-Xlinker", libdir]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed:\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose=True, ptxas_verbose="-v" in sys.argv)
    print(LIB)
