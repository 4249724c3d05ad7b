"""Build the CUDA library libtinylu.so in-tree for sm_103a.

Every (n, lanes-per-system) kernel family is its own translation unit
(csrc/tl_inst.cu compiled with -DTL_INST_N/-DTL_INST_T), so the build runs
in parallel on all host cores.  Objects are cached under _build/ keyed by a
hash of the sources and flags.

Spill gate: every unit is compiled with `-Xptxas -v`; its report is kept
beside the object and parsed after the build.  A kernel that spills
registers to local memory (spill stores or loads > 0) fails the build
unless it is on SPILL_ALLOW with at most the bytes listed there -- a silent
spill regression in a hot kernel would cost more than any tuning gains.
The parsed table (registers, stack frame, spills per kernel) is written to
_build/ptxas_report.txt.

The same build also links libtinylu_checked.so: the units of the
fixed-size and ragged solves (CHECKED_SOURCES) compiled with
-DTL_CHECK_BOUNDS, where every shared-memory index of the element-walk
solver is checked and a violation is counted in a device word instead of
being performed (tl_bounds.cuh); tests run it on small cases and expect no
violation.
"""
import concurrent.futures as cf
import hashlib
import os
import re
import shutil
import subprocess
import sys

PKG = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(PKG)
CSRC = os.path.join(PKG, "csrc")
INCLUDE = os.path.join(ROOT, "include")
BUILD = os.path.join(ROOT, "_build", "tinylu")
LIB = os.path.join(PKG, "libtinylu.so")
LIB_CHECKED = os.path.join(PKG, "libtinylu_checked.so")

ARCH = ["-gencode", "arch=compute_103a,code=sm_103a"]
NVCC_FLAGS = (["-O3", "-std=c++17", "-lineinfo", "-Xcompiler", "-fPIC", "--expt-relaxed-constexpr",
               "-Xptxas", "-v", "-I" + INCLUDE, "-I" + CSRC]
              + os.environ.get("TL_NVCC_FLAGS", "").split())
CHECK_FLAGS = ["-DTL_CHECK_BOUNDS=1"]

# Kernels allowed to spill, with the most spill bytes (stores, loads) each
# may use: (regex on the mangled name, max store bytes, max load bytes).
# Every other kernel must not spill at all.
SPILL_ALLOW = [
    # fused Newton kernels: the law's fields, the Jacobian and the register
    # LUpp of a point live across the iteration (255 registers); measured
    # faster than the shared-memory Newton kernel up to n = 24 all the same
    (r"k_newton_norton", 2048, 2048),
    (r"k_newton_tanh", 512, 512),
    (r"slow_tanh_solve", 256, 256),
    # LU-output register variants (getrf, gesv + factors) keep L in
    # registers as well; tuned dispatch runs the shared-memory solver there
    (r"k_factor_groupILi\d+ELi\d+ELi\d+ELi\d+ELb1E", 640, 640),
    (r"k_factor_groupILi23ELi8E", 16, 16),
    (r"k_fixup_thread|k_getrs_thread", 32, 32),
    (r"k_ragged_irILi1[34]ELi4E", 64, 64),
    # shared-memory solvers: ptxas parks a few addresses of the load and
    # store phases on the stack (the same with a higher register limit);
    # the refinement warp kernel at 64 registers (8 blocks per SM, measured
    # faster than 7 blocks without the spill)
    (r"k_smem_group|k_smem_ragged|k_smem_ir|k_ragged_persist", 32, 32),
]

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

# Units of the bounds-checked library: the C ABI, the shared-memory solvers
# (fixed-size and ragged, with the single persistent launch), the entry
# without allocation, the dispatcher and the peak probe.  The register
# kernels, mixed precision, Newton and the server are not in it.
CHECKED_SOURCES = ["tl_api.cu", "tl_inst_smem.cu", "tl_ragged.cu", "tl_noalloc.cu", "tl_autotune.cu", "tl_peak.cu"]

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


def _jobs(checked=False):
    hdr = _headers_digest()
    jobs = []
    if checked:
        for src in CHECKED_SOURCES:
            jobs.append((src, CHECK_FLAGS))
    else:
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
        stem = "_".join([os.path.splitext(src)[0]] + [d.split("=")[-1] for d in defs if "INST" in d])
        if checked:
            stem += "_checked"
        obj = os.path.join(BUILD, f"{stem}.{key}.o")
        out.append((path, defs, obj))
    return out


def _compile(nvcc, path, defs, obj, verbose):
    if os.path.exists(obj) and os.path.exists(obj + ".ptxas"):
        return obj, ""
    tmp = obj + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, *NVCC_FLAGS, *defs, "-c", path, "-o", tmp]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"nvcc failed: {' '.join(cmd)}\n{res.stdout}\n{res.stderr}")
    with open(obj + ".ptxas.tmp", "w") as fh:
        fh.write(res.stderr)
    os.replace(obj + ".ptxas.tmp", obj + ".ptxas")
    os.replace(tmp, obj)
    return obj, (res.stderr if verbose else "")


_FUNC = re.compile(r"Function properties for (\S+)")
_SPILL = re.compile(r"(\d+) bytes stack frame, (\d+) bytes spill stores, (\d+) bytes spill loads")


def ptxas_table(objs):
    """(kernel, registers, stack, spill stores, spill loads) from the ptxas
    reports of the objects (every entry function and device function)."""
    rows = {}
    for o in objs:
        try:
            text = open(o + ".ptxas").read()
        except OSError:
            continue
        func = entry = None
        for line in text.splitlines():
            m = _FUNC.search(line)
            if m:
                func = m.group(1)
                continue
            m = _SPILL.search(line)
            if m and func:
                st, ss, sl = (int(v) for v in m.groups())
                rows.setdefault(func, [None, 0, 0, 0])
                rows[func][1:] = [st, ss, sl]
                continue
            if "Compiling entry function" in line:
                entry = line.split("'")[1]
                continue
            m = re.search(r"Used (\d+) registers", line)
            if m and entry:
                rows.setdefault(entry, [None, 0, 0, 0])[0] = int(m.group(1))
    return sorted((k, *v) for k, v in rows.items())


def spill_gate(objs):
    """Raise when a kernel spills beyond SPILL_ALLOW; write the report."""
    table = ptxas_table(objs)
    bad = []
    with open(os.path.join(BUILD, "ptxas_report.txt"), "w") as fh:
        fh.write("kernel registers stack_bytes spill_store_bytes spill_load_bytes\n")
        for name, regs, st, ss, sl in table:
            fh.write(f"{name} {regs} {st} {ss} {sl}\n")
            if ss == 0 and sl == 0:
                continue
            allowed = [(a, b) for pat, a, b in SPILL_ALLOW if re.search(pat, name)]
            if not allowed or ss > allowed[0][0] or sl > allowed[0][1]:
                bad.append(f"{name}: {ss} B spill stores, {sl} B spill loads")
    if bad:
        raise RuntimeError("register spills (see SPILL_ALLOW in build.py):\n  " + "\n  ".join(bad))
    return table


def build(verbose=False, jobs=None) -> str:
    """Compile every kernel family and link libtinylu.so; returns its path."""
    nvcc = _nvcc()
    os.makedirs(BUILD, exist_ok=True)
    todo = _jobs()
    todo_checked = _jobs(checked=True)
    jobs = jobs or max(1, os.cpu_count() or 1)
    objs, objs_checked = [], []
    with cf.ThreadPoolExecutor(max_workers=jobs) as ex:
        # the slowest units first, so the pool's tail is short
        order = sorted(todo + todo_checked, key=lambda j: ("tl_inst_smem" not in j[0], "tl_ragged" not in j[0]))
        futs = {ex.submit(_compile, nvcc, p, d, o, verbose): o for p, d, o in order}
        done = {}
        for f in futs:
            obj, log = f.result()
            done[obj] = True
            if log:
                sys.stderr.write(log)
    objs = [o for _, _, o in todo]
    objs_checked = [o for _, _, o in todo_checked]
    spill_gate(objs + objs_checked)
    _link(nvcc, LIB, objs)
    _link(nvcc, LIB_CHECKED, objs_checked)
    return LIB


def _link(nvcc, lib, objs):
    newest = max(os.path.getmtime(o) for o in objs)
    if os.path.exists(lib) and os.path.getmtime(lib) >= newest and _objs_stamp_ok(lib, objs):
        return
    tmp = lib + f".tmp{os.getpid()}"
    cmd = [nvcc, *ARCH, "-shared", "-Xcompiler", "-fPIC", "-o", tmp, *objs, "-lpthread"]
    res = subprocess.run(cmd, capture_output=True, text=True)
    if res.returncode != 0:
        raise RuntimeError(f"link failed: {' '.join(cmd)}\n{res.stderr}")
    os.replace(tmp, lib)
    with open(lib + ".objs", "w") as fh:
        fh.write("\n".join(sorted(os.path.basename(o) for o in objs)))


def _objs_stamp_ok(lib, objs):
    stamp = lib + ".objs"
    if not os.path.exists(stamp):
        return False
    with open(stamp) as fh:
        return fh.read() == "\n".join(sorted(os.path.basename(o) for o in objs))


if __name__ == "__main__":
    print(build(verbose="-v" in sys.argv))
