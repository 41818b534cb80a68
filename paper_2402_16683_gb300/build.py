"""Build the in-tree CUDA library ``libnre.so`` for sm_103a with nvcc.

Every ``csrc/*.cu`` / ``csrc/*.cpp`` file is compiled in parallel to an object
under ``_build/`` and linked into ``paper_2402_16683_gb300/libnre.so``.
Usage: ``python -m paper_2402_16683_gb300.build [--force] [--verbose]``.
"""
import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(os.path.dirname(HERE), "_build")
LIB = os.path.join(HERE, "libnre.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    if not os.path.exists(cand):
        raise RuntimeError("nvcc not found; the CUDA toolkit is required to build libnre.so")
    return cand


def _sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _headers():
    inc = os.path.join(os.path.dirname(HERE), "include")
    hs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    hs += [os.path.join(inc, f) for f in os.listdir(inc) if f.endswith(".h")]
    return hs


def _stale(obj, src, headers):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(p) > t for p in [src] + headers)


def build(force=False, verbose=False, extra_flags=()):
    os.makedirs(BUILD, exist_ok=True)
    nv = nvcc()
    headers = _headers()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-O2",
                    "-I" + os.path.join(os.path.dirname(HERE), "include")] + list(extra_flags)
    if verbose:
        flags += ["-Xptxas", "-v"]
    jobs = []
    objs = []
    units = []
    for src in _sources():
        if os.path.basename(src) == "sweeps_inst.cu":
            # one object per (dtype, line length) so the sweep kernels build in parallel
            for t in ("float", "double"):
                for l2 in range(3, 13):
                    units.append((src, f"sweeps_{t}_{1 << l2}",
                                  [f"-DNRE_SWEEP_T={t}", f"-DNRE_SWEEP_L={1 << l2}"]))
        else:
            units.append((src, os.path.basename(src), []))
    for src, tag, defs in units:
        obj = os.path.join(BUILD, tag + ".o")
        objs.append(obj)
        if force or verbose or _stale(obj, src, headers):
            jobs.append([nv, "-c", src, "-o", obj] + flags + defs)

    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        return cmd, r

    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for cmd, r in ex.map(run, jobs):
                if verbose or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError("nvcc failed: " + " ".join(cmd))
    if jobs or not os.path.exists(LIB) or any(os.path.getmtime(o) > os.path.getmtime(LIB) for o in objs):
        cmd = [nv, "-shared", "-o", LIB] + objs + ARCH + ["-Xcompiler", "-fPIC"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            sys.stderr.write(r.stdout + r.stderr)
            raise RuntimeError("link failed: " + " ".join(cmd))
    return LIB


if __name__ == "__main__":
    build(force="--force" in sys.argv, verbose="--verbose" in sys.argv)
    print(LIB)
