"""Build the CUDA library ``_lib/libmatcha.so`` for sm_103a with nvcc.

Translation units compile in parallel; the shared object is linked with the
static CUDA runtime.  Build products are git-ignored.
"""
import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
OUT = os.path.join(HERE, "_lib", "libmatcha.so")
PROBE = os.path.join(HERE, "_lib", "libpeakprobe.so")
SOURCES = ["matcha_api.cu", "plan_tables.cu", "analyze.cu", "correlate.cu", "soft.cu", "newton.cu",
           "noalloc.cu", "backward.cu", "translate.cu", "pose6d.cu", "ball.cu",
           "correlate_tc.cu"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _deps():
    hdrs = [os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cuh", ".h"))]
    return hdrs + [os.path.join(HERE, "..", "include", "matcha.h")]


def _stale(target, deps):
    if not os.path.exists(target):
        return True
    t = os.path.getmtime(target)
    return any(os.path.getmtime(d) > t for d in deps)


def build(force=False, verbose=False, ptxas_v=False):
    os.makedirs(BUILD, exist_ok=True)
    os.makedirs(os.path.dirname(OUT), exist_ok=True)
    nvcc = _nvcc()
    hdeps = _deps()
    objs, jobs = [], []
    for s in SOURCES:
        src = os.path.join(CSRC, s)
        obj = os.path.join(BUILD, s.replace(".cu", ".o"))
        objs.append(obj)
        if force or _stale(obj, [src] + hdeps):
            cmd = [nvcc] + ARCH + FLAGS + (["-Xptxas", "-v"] if ptxas_v else []) + ["-c", src, "-o", obj]
            jobs.append(cmd)
    def run(cmd):
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("nvcc failed:\n" + " ".join(cmd) + "\n" + r.stdout + r.stderr)
        return r.stdout + r.stderr
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=min(len(jobs), os.cpu_count() or 4)) as ex:
            for log in ex.map(run, jobs):
                if verbose and log.strip():
                    print(log)
    if force or jobs or _stale(OUT, objs):
        tmp = OUT + ".tmp%d" % os.getpid()
        run([nvcc] + ARCH + ["-shared", "-o", tmp] + objs)
        os.replace(tmp, OUT)
    # the FP32 throughput probe the bench divides ALU work by (not part of the path)
    probe_src = os.path.join(CSRC, "peak_probe.cu")
    if force or _stale(PROBE, [probe_src]):
        run([nvcc] + ARCH + FLAGS + ["-shared", "-o", PROBE + ".tmp", probe_src])
        os.replace(PROBE + ".tmp", PROBE)
    # a C program using the library through its C ABI alone
    ex_src = os.path.join(HERE, "examples", "align_from_c.c")
    ex_out = os.path.join(HERE, "_lib", "align_from_c")
    if force or _stale(ex_out, [ex_src, OUT] + hdeps):
        cuda = os.path.dirname(os.path.dirname(nvcc)) if os.path.isabs(nvcc) else "/usr/local/cuda"
        libdir = os.path.join(HERE, "_lib")
        cudalib = next((d for d in (os.path.join(cuda, "lib64"), os.path.join(cuda, "lib"))
                        if os.path.isdir(d)), os.path.join(cuda, "lib64"))
        run(["gcc", "-O2", "-std=c11", "-o", ex_out + ".tmp", ex_src,
             "-I", os.path.join(HERE, "..", "include"), "-I", os.path.join(cuda, "include"),
             "-L", libdir, "-lmatcha", "-L", cudalib, "-lcudart",
             "-Wl,-rpath," + libdir, "-Wl,-rpath," + cudalib])
        os.replace(ex_out + ".tmp", ex_out)
    return OUT


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose=True, ptxas_v="-v" in sys.argv))
