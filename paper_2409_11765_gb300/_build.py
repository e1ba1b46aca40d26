"""Builds the engine's shared library in-tree with nvcc for sm_103a."""
import os
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(PKG, "csrc")
BUILD = os.path.join(PKG, "_build")
LIBDIR = os.path.join(PKG, "_lib")
LIB = os.path.join(LIBDIR, "libcmaes_gb300.so")
PROBE_LIB = os.path.join(LIBDIR, "libcmaes_probe.so")
INCLUDE = os.path.join(os.path.dirname(PKG), "include")
SOURCES = ["kernels_gen.cu", "kernels_eig.cu", "kernels_jacobi_cluster.cu", "kernels_mixed.cu",
           "kernels_eig_mixed.cu", "kernels_eig_big.cu", "kernels_eig_trd.cu", "kernels_eig_trd_bt.cu", "kernels_ozaki.cu", "capi.cu", "noalloc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-std=c++17", "--extended-lambda", "-O3", "-lineinfo", "-Xcompiler", "-fPIC",
         "-Xcompiler", "-O2"]


def _nvcc():
    for cand in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if cand and (os.path.isabs(cand) and os.path.exists(cand) or not os.path.isabs(cand)):
            return cand
    return "nvcc"


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files += [os.path.join(INCLUDE, f) for f in os.listdir(INCLUDE)]
    return files


def up_to_date():
    if not (os.path.exists(LIB) and os.path.exists(PROBE_LIB)):
        return False
    t = min(os.path.getmtime(LIB), os.path.getmtime(PROBE_LIB))
    return all(os.path.getmtime(f) <= t for f in _deps())


def build(force=False, verbose=False):
    """Compile the CUDA sources in parallel and link libcmaes_gb300.so and
    libcmaes_probe.so."""
    if not force and up_to_date():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(LIBDIR, exist_ok=True)
    nvcc = _nvcc()
    jobs = []
    objs = []
    for src in SOURCES:
        obj = os.path.join(BUILD, src.replace(".cu", ".o"))
        objs.append(obj)
        jobs.append((src, [nvcc, *FLAGS, *ARCH, "-I", INCLUDE, "-c", os.path.join(CSRC, src),
                           "-o", obj]))
    jobs.append(("probe.cu", [nvcc, *FLAGS, *ARCH, "-I", INCLUDE, "-shared", "-o",
                              PROBE_LIB + ".tmp", os.path.join(CSRC, "probe.cu")]))
    procs = []
    for src, cmd in jobs:
        if verbose:
            print(" ".join(cmd), file=sys.stderr)
        procs.append((src, subprocess.Popen(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)))
    errors = []
    for src, p in procs:
        out, _ = p.communicate()
        if p.returncode != 0:
            errors.append("%s:\n%s" % (src, out.decode(errors="replace")))
    if errors:
        raise RuntimeError("nvcc failed\n" + "\n".join(errors))
    os.replace(PROBE_LIB + ".tmp", PROBE_LIB)
    tmp = LIB + ".tmp"
    cmd = [nvcc, "-shared", *ARCH, "-o", tmp, *objs, "-lcudart"]
    r = subprocess.run(cmd, stdout=subprocess.PIPE, stderr=subprocess.STDOUT)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n" + r.stdout.decode(errors="replace"))
    os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True))
