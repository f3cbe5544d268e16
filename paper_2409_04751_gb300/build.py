"""Build the sm_103a CUDA library libfgs.so in-tree (paper_2409_04751_gb300/_build/).

Each .cu file is compiled in parallel with nvcc for sm_103a only, then linked into one shared
library exporting the C ABI of include/fgs.h. No cmake; the whole build takes well under a
minute. The same sources compiled with -DFGS_CHECK=1 give the checked build libfgs_check.so
(_build/check/): the same ABI with every index read from memory compared with its buffer's size
before use (FGS_ERR_BOUNDS instead of an access out of bounds), for debugging.
"""
import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libfgs.so")
CHECK_DIR = os.path.join(BUILD_DIR, "check")
CHECK_LIB_PATH = os.path.join(CHECK_DIR, "libfgs_check.so")
SOURCES = ["api.cu", "preprocess.cu", "binsort.cu", "onesweep.cu", "raster.cu", "noalloc.cu",
           "train.cu"]
HEADERS = ["fgs_internal.cuh", "scan.cuh", os.path.join("..", "..", "include", "fgs.h")]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", "nvcc"):
        if c and (os.path.isabs(c) and os.path.exists(c) or not os.path.isabs(c)):
            return c
    return "nvcc"


def _stale(outputs, inputs):
    if not all(os.path.exists(o) for o in outputs):
        return True
    newest = max(os.path.getmtime(i) for i in inputs)
    return min(os.path.getmtime(o) for o in outputs) < newest


def _variants(check):
    """(library path, object directory, extra nvcc flags) of the builds asked for."""
    out = [(LIB_PATH, BUILD_DIR, [])]
    if check:
        out.append((CHECK_LIB_PATH, CHECK_DIR, ["-DFGS_CHECK=1"]))
    return out


def build(force: bool = False, verbose: bool = False, extra_flags=(), check: bool = False) -> str:
    """Build libfgs.so (and with check=True also libfgs_check.so, all objects compiled in one
    parallel batch); returns the path of libfgs.so."""
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.normpath(os.path.join(CSRC, h)) for h in HEADERS]
    inputs = srcs + hdrs + [os.path.abspath(__file__)]
    todo = [v for v in _variants(check) if force or _stale([v[0]], inputs)]
    if not todo:
        return LIB_PATH
    nvcc = _nvcc()
    base = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                   "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"] + list(extra_flags)
    if verbose:
        base += ["-Xptxas", "-v"]
    jobs = []
    for lib, odir, vflags in todo:
        os.makedirs(odir, exist_ok=True)
        for s in SOURCES:
            jobs.append((os.path.join(CSRC, s), os.path.join(odir, s.replace(".cu", ".o")), vflags))

    def compile_one(job):
        src, obj, vflags = job
        cmd = [nvcc] + base + vflags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
        logs = list(ex.map(compile_one, jobs))
    if verbose:
        for lg in logs:
            print(lg)
    for lib, odir, _ in todo:
        objs = [os.path.join(odir, s.replace(".cu", ".o")) for s in SOURCES]
        tmp = lib + f".{os.getpid()}.tmp"
        cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
        os.replace(tmp, lib)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv, check="--check" in sys.argv))
