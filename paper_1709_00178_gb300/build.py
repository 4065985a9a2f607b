"""Builds the CUDA library ``libpyrit.so`` in-tree for sm_103a (GB300).

Every translation unit under ``csrc/`` is compiled by nvcc in parallel into ``_build/`` and linked
into ``paper_1709_00178_gb300/libpyrit.so`` next to this file. Rebuilds only what changed.

The device headers that plan-specialised networks are compiled against at run time (NVRTC has no
file system view of ``csrc/``) are embedded into the library as string literals: this script
writes them to ``_build/jit_sources.inc``, which ``csrc/net_jit.cpp`` includes.
"""
import concurrent.futures as cf
import glob
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libpyrit.so")
INCLUDE = os.path.join(os.path.dirname(HERE), "include")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2,-fvisibility=hidden", "-I" + INCLUDE, "-I" + CSRC,
         "-I" + BUILD]
# What the run-time compiler sees, in include order: the shared plain-data types, the PTX wrappers
# and the staged pipeline.
JIT_HEADERS = ("ring_abi.h", "ptx.cuh", "ring_staged.cuh")
_DELIM = "PYRIT_SRC"


def _write_jit_sources():
    """Writes _build/jit_sources.inc (only when its text changes, to keep rebuilds minimal)."""
    names, texts = [], []
    for name in JIT_HEADERS:
        with open(os.path.join(CSRC, name)) as f:
            text = f.read()
        if ")" + _DELIM + '"' in text:
            raise RuntimeError("%s contains the raw-string delimiter" % name)
        names.append('"%s"' % name)
        texts.append('R"%s(%s)%s"' % (_DELIM, text, _DELIM))
    body = ("// Generated by build.py from csrc/{%s}: the device sources of the run-time compiler.\n"
            "static const int kJitHeaderCount = %d;\n"
            "static const char* const kJitHeaderNames[] = {%s};\n"
            "static const char* const kJitHeaders[] = {\n%s};\n") % (
                ", ".join(JIT_HEADERS), len(JIT_HEADERS), ", ".join(names), ",\n".join(texts))
    path = os.path.join(BUILD, "jit_sources.inc")
    if os.path.exists(path):
        with open(path) as f:
            if f.read() == body:
                return
    with open(path, "w") as f:
        f.write(body)


def _deps_mtime():
    files = glob.glob(os.path.join(CSRC, "*.h")) + glob.glob(os.path.join(CSRC, "*.cuh")) + \
        glob.glob(os.path.join(INCLUDE, "*.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src, obj, verbose):
    cmd = [NVCC] + ARCH + FLAGS + (["-Xptxas", "-v"] if verbose else []) + ["-c", src, "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s%s" % (src, r.stdout, r.stderr))
    return r.stderr


def build(force: bool = False, verbose: bool = False) -> str:
    os.makedirs(BUILD, exist_ok=True)
    _write_jit_sources()
    srcs = sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))
    dep = _deps_mtime()
    jobs = []
    objs = []
    for s in srcs:
        o = os.path.join(BUILD, os.path.basename(s) + ".o")
        objs.append(o)
        if force or not os.path.exists(o) or os.path.getmtime(o) < max(os.path.getmtime(s), dep):
            jobs.append((s, o))
    with cf.ThreadPoolExecutor(max_workers=max(1, min(len(jobs), os.cpu_count() or 4))) as ex:
        for out in ex.map(lambda so: _compile(so[0], so[1], verbose), jobs):
            if verbose and out:
                print(out)
    if force or jobs or not os.path.exists(LIB) or os.path.getmtime(LIB) < max(os.path.getmtime(o) for o in objs):
        tmp = LIB + ".tmp.%d" % os.getpid()
        cmd = [NVCC] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart", "-lnvrtc"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
