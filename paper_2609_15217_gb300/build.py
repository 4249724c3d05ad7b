"""Build the CUDA library libtinylu.so in-tree for sm_103a.

Every (n, lanes-per-system) kernel family is its own translation unit
(csrc/tl_inst.cu compiled with -DTL_INST_N/-DTL_INST_T), so the build runs
in parallel on all host cores.  Objects are cached under _build/ keyed by a
hash of the sources and flags.
"""
import concurrent.futures as cf
import hashlib
import os
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "tinylu")
LIB = os.path.join(PKG, "libtinylu.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = ["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
              "-I" + INCLUDE, "-I" + CSRC] + os.environ.get("TL_NVCC_FLAGS", "").split()

# (n, lanes per system) kernel families compiled into the library.
#   lanes = 1: one thread per system, matrix in registers (n <= 9)
#   lanes > 1: row-cyclic sub-warp groups
KERNEL_FAMILIES = (
    [(n, 1) for n in range(1, 10)]
    + [(n, 2) for n in range(10, 13)]
    + [(n, 4) for n in range(13, 17)]
    + [(n, 8) for n in range(17, 25)]
    + [(n, 16) for n in range(25, 33)]
)

# (n, lanes per system) families of the mixed-precision (binary32 factor,
# binary64 refinement) ragged kernel; binary32 rows take half the registers,
# so one thread per system reaches further.
IR_FAMILIES = (
    [(n, 1) for n in range(1, 11)]
    + [(n, 4) for n in range(11, 17)]
    + [(n, 8) for n in range(17, 25)]
    + [(n, 16) for n in range(25, 33)]
)

# (n, lanes per point) of the sub-warp tanh-law Newton kernel (n >= 10;
# smaller n run one thread per point).
NEWTON_GROUP_FAMILIES = [(n, t) for n, t in KERNEL_FAMILIES if n >= 10]

PLAIN_SOURCES = ["tl_api.cu", "tl_newton.cu", "tl_newton_cpu_driven.cu", "tl_ragged.cu", "tl_noalloc.cu", "tl_inst_smem.cu", "tl_autotune.cu", "tl_server.cu", "tl_newton_smem.cu", "tl_peak.cu"]


def _nvcc():
    for c in (os.environ.get("NVCC"), "/usr/local/cuda/bin/nvcc", shutil.which("nvcc")):
        if c and os.path.exists(c):
            return c
    raise RuntimeError("nvcc not found")


def _headers_digest():
    h = hashlib.sha256()
    for d in (CSRC, INCLUDE):
        for f in sorted(os.listdir(d)):
            if f.endswith((".h", ".cuh", ".inc")):
                with open(os.path.join(d, f), "rb") as fh:
                    h.update(f.encode() + fh.read())
    return h.hexdigest()


def _jobs():
    hdr = _headers_digest()
    jobs = []
    for src in PLAIN_SOURCES:
        jobs.append((src, []))
    for n, t in KERNEL_FAMILIES:
        jobs.append(("tl_inst.cu", [f"-DTL_INST_N={n}", f"-DTL_INST_T={t}"]))
    for n, t in IR_FAMILIES:
        jobs.append(("tl_inst_ir.cu", [f"-DTL_INST_N={n}", f"-DTL_INST_T={t}"]))
    for n, t in NEWTON_GROUP_FAMILIES:
        jobs.append(("tl_inst_newton.cu", [f"-DTL_INST_N={n}", f"-DTL_INST_T={t}"]))
    out = []
    for src, defs in jobs:
        path = os.path.join(CSRC, src)
        with open(path, "rb") as fh:
            body = fh.read()
        key = hashlib.sha256(body + hdr.encode() + " ".join(NVCC_FLAGS + ARCH + defs).encode()).hexdigest()[:16]
        stem = "_".join([os.path.splitext(src)[0]] + [d.split("=")[-1] for d in defs])
        obj = os.path.join(BUILD, f"{stem}.{key}.o")
        out.append((path, defs, obj))
    return out


def _compile(nvcc, path, defs, obj, verbose):
    if os.path.exists(obj):
        return obj, ""
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-c", path, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    os.replace(tmp, obj)
    return obj, (res.stderr if verbose else "")


def build(verbose=False, jobs=None) -> str:
    """Compile every kernel family and link libtinylu.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    todo = _jobs()
    jobs = jobs or max(1, os.cpu_count() or 1)
    objs = []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        futs = [ex.submit(_compile, nvcc, p, d, o, verbose) for p, d, o in todo]
        for f in futs:
            obj, log = f.result()
            objs.append(obj)
            if log:
                sys.stderr.write(log)
    newest = max(os.path.getmtime(o) for o in objs)
    if os.path.exists(LIB) and os.path.getmtime(LIB) >= newest and _objs_stamp_ok(objs):
        return LIB
    tmp = LIB + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stderr}")
    os.replace(tmp, LIB)
    with open(LIB + ".objs", "w") as fh:
        fh.write("\n".join(sorted(os.path.basename(o) for o in objs)))
    return LIB


def _objs_stamp_ok(objs):
    stamp = LIB + ".objs"
    if not os.path.exists(stamp):
        return False
    with open(stamp) as fh:
        return fh.read() == "\n".join(sorted(os.path.basename(o) for o in objs))


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
