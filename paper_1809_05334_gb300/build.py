"""Build the CUDA library libvie.so in-tree with nvcc for sm_103a (GB300).

Usage: python -m paper_1809_05334_gb300.build [--force]
The translation units are compiled in parallel; the library is linked with
OpenMP (host topology build).  Nothing is installed outside this directory.
VIE_NVCC_DEFINES (optional, space-separated -D flags) overrides the schedule
constants that have a compile-time default, for sweeps, e.g.
    VIE_NVCC_DEFINES="-DVIE_GJ_RESERVE_WIDE=24" python -m paper_1809_05334_gb300.build --force
(VIE_SPLIT_NORMAL, VIE_SPLIT_OBLIQUE, VIE_FAR_N_MINB, VIE_FAR_O_MINB,
VIE_GJ_RESERVE, VIE_GJ_RESERVE_WIDE).  The defines are part of the staleness
check: a build with other defines rebuilds.
"""
import concurrent.futures
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "libvie.so")
BUILD = os.path.join(HERE, "_build")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
SOURCES = ["api.cu", "fill.cu", "linalg.cu", "post.cu", "topology.cpp", "rules.cpp", "server.cpp",
           "ewald_tables.cpp", "blocks.cpp"]


def _nvcc():
    path = shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(path):
        raise RuntimeError("nvcc not found: the CUDA toolkit is required to build libvie.so")
    return path


def _defines():
    flags = os.environ.get("VIE_NVCC_DEFINES", "").split()
    for f in flags:
        if not f.startswith("-DVIE_"):
            raise RuntimeError("VIE_NVCC_DEFINES takes -DVIE_... flags only, got %r" % f)
    return flags


STAMP = os.path.join(HERE, "_build", "defines.txt")


def _stale():
    if not os.path.exists(OUT):
        return True
    old = open(STAMP).read() if os.path.exists(STAMP) else ""
    if old != " ".join(_defines()):
        return True
    t = os.path.getmtime(OUT)
    deps = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    deps.append(os.path.join(HERE, "..", "include", "vie.h"))
    return any(os.path.getmtime(d) > t for d in deps if os.path.exists(d))


def build(force=False, verbose=False):
    if not force and not _stale():
        return OUT
    os.makedirs(BUILD, exist_ok=True)
    nvcc = _nvcc()
    common = ["-O3", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-fopenmp", "-lineinfo"] + _defines()

    def compile_one(src):
        obj = os.path.join(BUILD, src + ".o")
        cmd = [nvcc, *ARCH, *common, "-c", os.path.join(CSRC, src), "-o", obj]
        if src.endswith(".cu"):
            cmd += ["-Xptxas", "-v"] if verbose else []
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed for %s:\n%s" % (src, r.stderr[-6000:]))
        return obj, r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(SOURCES)) as ex:
        results = list(ex.map(compile_one, SOURCES))
    objs = [o for o, _ in results]
    if verbose:
        for _, log in results:
            sys.stderr.write(log)
    tmp = OUT + ".tmp"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-Xcompiler", "-fopenmp", "-lgomp"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr[-6000:])
    os.replace(tmp, OUT)
    with open(STAMP, "w") as f:
        f.write(" ".join(_defines()))
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
