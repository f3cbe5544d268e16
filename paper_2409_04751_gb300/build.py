"""Build the sm_103a CUDA library libfgs.so in-tree (paper_2409_04751_gb300/_build/).

Each .cu file is compiled in parallel with nvcc for sm_103a only, then linked into one shared
library exporting the C ABI of include/fgs.h. No cmake; the whole build takes well under a
minute.
"""
import concurrent.futures
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD_DIR = os.path.join(HERE, "_build")
LIB_PATH = os.path.join(BUILD_DIR, "libfgs.so")
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


def build(force: bool = False, verbose: bool = False, extra_flags=()) -> str:
    os.makedirs(BUILD_DIR, exist_ok=True)
    srcs = [os.path.join(CSRC, s) for s in SOURCES]
    hdrs = [os.path.normpath(os.path.join(CSRC, h)) for h in HEADERS]
    objs = [os.path.join(BUILD_DIR, s.replace(".cu", ".o")) for s in SOURCES]
    if not force and not _stale([LIB_PATH], srcs + hdrs + [os.path.abspath(__file__)]):
        return LIB_PATH
    nvcc = _nvcc()
    flags = ARCH + ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC",
                    "--expt-relaxed-constexpr", "-Xptxas", "-warn-spills"] + list(extra_flags)
    if verbose:
        flags += ["-Xptxas", "-v"]

    def compile_one(pair):
        src, obj = pair
        cmd = [nvcc] + flags + ["-c", src, "-o", obj]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stdout}\n{r.stderr}")
        return r.stderr

    with concurrent.futures.ThreadPoolExecutor(max_workers=len(srcs)) as ex:
        logs = list(ex.map(compile_one, zip(srcs, objs)))
    if verbose:
        for lg in logs:
            print(lg)
    tmp = LIB_PATH + f".{os.getpid()}.tmp"
    cmd = [nvcc] + ARCH + ["-shared", "-o", tmp] + objs + ["-lcudart_static"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stdout}\n{r.stderr}")
    os.replace(tmp, LIB_PATH)
    return LIB_PATH


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
