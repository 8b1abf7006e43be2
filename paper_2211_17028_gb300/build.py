"""Build libnqs.so in-tree: every translation unit of csrc/ with nvcc for
sm_103a, compiled in parallel, then linked with the static CUDA runtime."""

import concurrent.futures as cf
import os
import shutil
import subprocess
import sys

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
OUT = os.path.join(HERE, "_build")
LIB = os.path.join(HERE, "libnqs.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]


def nvcc():
    cand = os.environ.get("NVCC") or shutil.which("nvcc") or "/usr/local/cuda/bin/nvcc"
    return cand


def sources():
    return sorted(os.path.join(CSRC, f) for f in os.listdir(CSRC) if f.endswith((".cu", ".cpp")))


def _includes(path, seen):
    """The quoted #include files that `path` pulls in, recursively."""
    try:
        lines = open(path).read().splitlines()
    except OSError:
        return seen
    for ln in lines:
        ln = ln.strip()
        if ln.startswith("#include \""):
            dep = os.path.normpath(os.path.join(os.path.dirname(path), ln.split('"')[1]))
            if dep not in seen and os.path.exists(dep):
                seen.add(dep)
                _includes(dep, seen)
    return seen


def _compile(src, extra):
    obj = os.path.join(OUT, os.path.basename(src) + ".o")
    headers = sorted(_includes(src, set()))
    newest = max(os.path.getmtime(p) for p in headers + [src])
    if os.path.exists(obj) and os.path.getmtime(obj) >= newest and not extra.get("force"):
        return obj
    cmd = [nvcc(), "-c", src, "-o", obj, "-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC",
           "-Xcompiler", "-O2", "--expt-relaxed-constexpr"] + ARCH
    if os.path.basename(src).startswith("kernels_sweep_s"):
        # one kernel pair per unit: below nvcc's default compression threshold
        cmd.append("--compress-mode=size")
    if extra.get("verbose_ptxas") and src.endswith(".cu"):
        cmd.append("-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc failed for %s:\n%s\n%s" % (src, r.stdout, r.stderr))
    if extra.get("verbose_ptxas"):
        sys.stderr.write(r.stderr)
    return obj


def build(force=False, verbose_ptxas=False):
    os.makedirs(OUT, exist_ok=True)
    srcs = sources()
    extra = {"force": force, "verbose_ptxas": verbose_ptxas}
    with cf.ThreadPoolExecutor(max_workers=min(8, len(srcs))) as ex:
        objs = list(ex.map(lambda s: _compile(s, extra), srcs))
    newest = max(os.path.getmtime(o) for o in objs)
    if force or not os.path.exists(LIB) or os.path.getmtime(LIB) < newest:
        tmp = LIB + ".tmp%d" % os.getpid()
        cmd = [nvcc(), "-shared", "-o", tmp] + objs + ARCH + ["-cudart", "static", "-ldl", "-lpthread"]
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError("link failed:\n%s\n%s" % (r.stdout, r.stderr))
        os.replace(tmp, LIB)
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose_ptxas="-v" in sys.argv))
