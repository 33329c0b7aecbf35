"""Build the sm_103a shared library ``libns_gb300.so`` in-tree.

The translation units compile in parallel (the host library and one
instantiation of the per-dimension kernels for each register class), then
nvcc links them with the static CUDA runtime.  Objects go to ``_build/``.
"""
import concurrent.futures as cf
import os
import subprocess

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
ROOT = os.path.dirname(HERE)
BUILD = os.path.join(ROOT, "_build")
LIB = os.path.join(HERE, "libns_gb300.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr"]
CLASSES = (2, 4, 6, 8, 10, 12, 16, 20, 24, 28, 32)


def _sources():
    out = [(os.path.join(CSRC, "ns_lib.cu"), os.path.join(BUILD, "ns_lib.o"), []),
           (os.path.join(CSRC, "ns_mlp.cu"), os.path.join(BUILD, "ns_mlp.o"), [])]
    for d in CLASSES:
        out.append((os.path.join(CSRC, "ns_inst.cu"), os.path.join(BUILD, f"ns_inst_{d}.o"),
                    [f"-DNS_DMAX={d}"]))
    return out


def _deps():
    files = [os.path.join(CSRC, f) for f in os.listdir(CSRC)]
    files.append(os.path.join(ROOT, "include", "ns_gb300.h"))
    return max(os.path.getmtime(f) for f in files)


def _compile(src, obj, extra, nvcc, verbose):
    cmd = [nvcc, *ARCH, *FLAGS, *extra, "-c", src, "-o", obj]
    if os.environ.get("NS_RUN_MINB"):
        cmd.insert(1, "-DNS_RUN_MINB=" + str(int(os.environ["NS_RUN_MINB"])))
    if os.environ.get("NS_RUN_MAXNREG"):
        cmd.insert(1, "-DNS_RUN_MAXNREG=" + str(int(os.environ["NS_RUN_MAXNREG"])))
    if verbose:
        cmd.insert(1, "-Xptxas=-v")
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"nvcc failed for {os.path.basename(obj)}:\n{r.stderr}")
    return r.stderr


def build(force=False, verbose=False):
    """Compile (if stale) and return the path of libns_gb300.so."""
    if not force and os.path.exists(LIB) and os.path.getmtime(LIB) >= _deps():
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    nvcc = os.environ.get("NVCC", "nvcc")
    logs = []
    workers = max(2, min(len(CLASSES) + 1, os.cpu_count() or 4))
    with cf.ThreadPoolExecutor(max_workers=workers) as ex:
        futs = [ex.submit(_compile, s, o, e, nvcc, verbose) for s, o, e in _sources()]
        for f in futs:
            logs.append(f.result())
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-o", tmp] + [o for _, o, _ in _sources()]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError("nvcc link failed:\n" + r.stderr)
    os.replace(tmp, LIB)
    if verbose:
        print("\n".join(logs))
    return LIB


if __name__ == "__main__":
    import sys
    print(build(force=True, verbose="-v" in sys.argv))
