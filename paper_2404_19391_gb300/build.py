"""Builds libzsmiles.so in-tree (sm_103a only) from csrc/*.cu with nvcc, one process per file."""
from __future__ import annotations

import glob
import os
import platform
import subprocess
import sys
import time
from concurrent.futures import ThreadPoolExecutor

HERE = os.path.dirname(os.path.abspath(__file__))
CSRC = os.path.join(HERE, "csrc")
BUILD = os.path.join(HERE, "_build")
LIB = os.path.join(BUILD, "libzsmiles.so")
ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC = os.environ.get("NVCC", "nvcc")
FLAGS = ["-O3", "-lineinfo", "-std=c++17", "-Xcompiler", "-fPIC", "-Xcompiler", "-O2"]


def _sources():
    return sorted(glob.glob(os.path.join(CSRC, "*.cu")) + glob.glob(os.path.join(CSRC, "*.cpp")))


def _stale() -> bool:
    if not os.path.exists(LIB):
        return True
    t = os.path.getmtime(LIB)
    deps = _sources() + glob.glob(os.path.join(CSRC, "*.cuh")) + glob.glob(os.path.join(CSRC, "*.h")) + \
        [os.path.join(os.path.dirname(HERE), "include", "zsmiles.h"), __file__]
    return any(os.path.getmtime(p) > t for p in deps)


def _nvcc_version() -> str:
    try:
        r = subprocess.run([NVCC, "--version"], capture_output=True, text=True)
        lines = [ln for ln in r.stdout.splitlines() if "release" in ln]
        return lines[-1].strip() if lines else r.stdout.strip().splitlines()[-1]
    except OSError as e:
        return f"unavailable ({e})"


def _log(msg: str) -> None:
    """One line to stderr and to _build/build_info.txt, so a run's record shows how the library came to be."""
    line = f"[zsmiles build] {msg}"
    sys.stderr.write(line + "\n")
    try:
        os.makedirs(BUILD, exist_ok=True)
        with open(os.path.join(BUILD, "build_info.txt"), "a") as f:
            f.write(time.strftime("%Y-%m-%dT%H:%M:%S ") + line + "\n")
    except OSError:
        pass


def build(force: bool = False, verbose: bool = False) -> str:
    if not force and not _stale():
        _log(f"reused {LIB} (newer than every source; host {platform.machine()})")
        return LIB
    os.makedirs(BUILD, exist_ok=True)
    t0 = time.time()
    objs = []

    def compile_one(src):
        obj = os.path.join(BUILD, os.path.basename(src) + ".o")
        cmd = [NVCC, *ARCH, *FLAGS, "-c", src, "-o", obj]
        if verbose:
            cmd.insert(1, "-Xptxas=-v")
        r = subprocess.run(cmd, capture_output=True, text=True)
        if r.returncode != 0:
            raise RuntimeError(f"nvcc failed for {src}:\n{r.stderr}")
        if verbose:
            sys.stderr.write(r.stderr)
        return obj

    with ThreadPoolExecutor(max_workers=max(1, min(8, os.cpu_count() or 1))) as ex:
        objs = list(ex.map(compile_one, _sources()))
    tmp = LIB + f".{os.getpid()}.tmp"
    cmd = [NVCC, *ARCH, "-shared", "-o", tmp, *objs, "-lpthread"]
    r = subprocess.run(cmd, capture_output=True, text=True)
    if r.returncode != 0:
        raise RuntimeError(f"link failed:\n{r.stderr}")
    os.replace(tmp, LIB)
    _log(f"compiled {len(objs)} sources on {platform.machine()} with nvcc {_nvcc_version()} "
         f"{' '.join(ARCH)} {' '.join(FLAGS)} in {time.time() - t0:.1f} s -> {LIB}")
    return LIB


if __name__ == "__main__":
    print(build(force="--force" in sys.argv, verbose="-v" in sys.argv))
