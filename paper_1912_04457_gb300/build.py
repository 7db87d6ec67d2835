"""Build libbz.so (the CUDA library behind include/bz.h) for sm_103a, in tree.

Each translation unit is compiled in parallel with nvcc; the FP64 collision
path, the transport kernels and the host layer are compiled without FMA
contraction (-fmad=false on the device, -ffp-contract=off on the host) so
their arithmetic is exactly the written formula.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(HERE)
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(OUT, "libbz.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]

# (source, extra flags)
UNITS = [
    ("k_collide_f64.cu", ["-fmad=false"]),
    ("k_collide_f32.cu", ["-use_fast_math"]),
    ("k_transport.cu", ["-fmad=false"]),
    ("k_mlp.cu", []),
    ("bz_api.cu", ["-fmad=false"]),
    ("bz_static.cu", ["-fmad=false"]),
]


def nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _compile(src, extra, out=OUT):
    obj = os.path.join(out, os.path.splitext(src)[0] + ".o")
    cmd = [nvcc(), *ARCH, "-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC,-ffp-contract=off",
           "-I", os.path.join(ROOT, "include"), *extra, "-c", os.path.join(CSRC, src), "-o", obj]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, " ".join(cmd), r.stderr))
    return obj


def _stale():
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    for d in (CSRC, os.path.join(ROOT, "include")):
        for f in os.listdir(d):
            if os.path.getmtime(os.path.join(d, f)) > t:
                return True
    return False


def build(force: bool = False, out_dir: str = None, extra=(), unit_extra=None) -> str:
    """Builds libbz.so into out_dir (default: the in-tree _build).  `extra`
    adds nvcc flags to every unit, `unit_extra` maps a source to flags that
    replace its own."""
    out = out_dir or OUT
    lib = os.path.join(out, "libbz.so")
    if not force and out == OUT and not _stale():
        return LIB
    os.makedirs(out, exist_ok=True)
    units = [(src, list((unit_extra or {}).get(src, fl)) + list(extra)) for src, fl in UNITS]
    with cf.ThreadPoolExecutor(max_workers=len(units)) as ex:
        objs = list(ex.map(lambda u: _compile(u[0], u[1], out), units))
    tmp = lib + ".tmp.%d" % os.getpid()
    cmd = [nvcc(), *ARCH, "-shared", "-o", tmp, *objs]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("link failed:\n%s" % r.stderr)
    os.replace(tmp, lib)
    return lib


if __name__ == "__main__":
    print(build(force=True))
