"""Build libffp.so in-tree with nvcc for sm_103a (one -gencode), compiling the
translation units in parallel.  No torch, no cmake: plain nvcc + a thread pool."""
from __future__ import annotations

import concurrent.futures as cf
import os
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libffp.so")
SOURCES = ["ffp_api.cu", "ffp_ops.cu", "ffp_dispatch.cu", "ffp_setup_a.cu", "ffp_setup_b.cu",
           "ffp_setup_c.cu", "ffp_setup_d.cu", "ffp_setup_e.cu", "ffp_apply_f64.cu", "ffp_apply_f32.cu",
           "ffp_apply_bf16.cu", "ffp_ilu.cu", "ffp_batch.cu", "ffp_net.cu", "ffp_lanczos.cu"]
HEADERS = ["ffp_internal.cuh", "ffp_plane.cuh", "ffp_kernels.h", "ffp_setup.cuh", "ffp_apply.cuh",
           "ffp_vecops.cuh"]
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _nvcc():
    cand = os.path.join(os.environ.get("CUDA_HOME", "/usr/local/cuda"), "bin", "nvcc")
    return cand if os.path.exists(cand) else "nvcc"


def _stale(obj, deps):
    if not os.path.exists(obj):
        return True
    t = os.path.getmtime(obj)
    return any(os.path.getmtime(d) > t for d in deps)


def build(verbose: bool = False, ptxas_info: bool = False, force: bool = False,
          profile: bool = False) -> str:
    """Compile libffp.so (or, with profile=True, libffp_profile.so: the same
    library with -DFFP_STEP_PROFILE, whose FP32 apply records a clock64 budget
    of its line steps, read by ffp_step_profile(); see profile_steps.py).
    Returns the library path."""
    build_dir = BUILD + ("_profile" if profile else "")
    lib_path = LIB.replace("libffp.so", "libffp_profile.so") if profile else LIB
    extra = ["-DFFP_STEP_PROFILE"] if profile else []
    os.makedirs(build_dir, exist_ok=True)
    nvcc = _nvcc()
    hdrs = [os.path.join(CSRC, h) for h in HEADERS] + [
        os.path.join(HERE, "..", "include", "ffp.h")]
    jobs = []
    for src in SOURCES:
        s = os.path.join(CSRC, src)
        o = os.path.join(build_dir, src.replace(".cu", ".o"))
        if force or _stale(o, [s] + hdrs):
            cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", s, "-o", o]
            if ptxas_info:
                cmd.insert(1, "-Xptxas=-v")
            jobs.append((src, cmd))
    def run(job):
        src, cmd = job
        r = subprocess.run(cmd, capture_output=True, text=True)
        return src, r
    if jobs:
        with cf.ThreadPoolExecutor(max_workers=len(jobs)) as ex:
            for src, r in ex.map(run, jobs):
                if verbose or ptxas_info or r.returncode != 0:
                    sys.stderr.write(r.stdout + r.stderr)
                if r.returncode != 0:
                    raise RuntimeError(f"nvcc failed on {src}")
    objs = [os.path.join(build_dir, s.replace(".cu", ".o")) for s in SOURCES]
    if force or jobs or _stale(lib_path, objs):
        tmp = lib_path + f".tmp{os.getpid()}"
        subprocess.check_call([nvcc, *ARCH, "-shared", "-o", tmp, *objs, "-lcudart"])
        os.replace(tmp, lib_path)
    return lib_path


if __name__ == "__main__":
    print(build(verbose=True, ptxas_info="-v" in sys.argv, force="-f" in sys.argv,
                profile="--profile" in sys.argv))
