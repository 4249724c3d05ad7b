"""Host-side checks that need no GPU:
  * the C-ABI library loads and exports every function include/tinylu.h
    declares, and the ctypes binding exposes the same names;
  * the product package never imports the oracle;
  * the multi-rank logic of the benchmark (independent per-rank batches,
    job time = max over ranks) on two gloo processes.
"""
import os
import re
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
HEADER = os.path.join(ROOT, "include", "tinylu.h")


def header_functions():
    text = open(HEADER).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(tl_[a-z0-9_]+)\s*\(", text)))


def _library():
    from paper_2609_15217_gb300 import build as B
    if not os.path.exists(B.LIB):
        try:
            B._nvcc()
        except RuntimeError:
            pytest.skip("no nvcc to build the library")
        B.build()
    import ctypes
    return ctypes.CDLL(B.LIB)


def test_library_exports_every_declared_function():
    names = header_functions()
    assert "tl_gesv_batched" in names and "tl_newton_integrate" in names and len(names) >= 12
    lib = _library()
    missing = [n for n in names if not hasattr(lib, n)]
    assert not missing, missing


def test_binding_has_the_same_names():
    _library()
    from paper_2609_15217_gb300 import tinylu
    missing = [n for n in header_functions() if not callable(getattr(tinylu, n, None))]
    assert not missing, missing


def test_status_strings_without_gpu():
    lib = _library()
    import ctypes
    lib.tl_status_string.restype = ctypes.c_char_p
    for code in (0, -1, -2, -3, -4, -5, 7):
        assert lib.tl_status_string(code)
    lib.tl_last_bad_arg.restype = ctypes.c_int
    assert lib.tl_last_bad_arg(None) == 0


def test_product_never_imports_the_oracle():
    pkg = os.path.join(ROOT, "paper_2609_15217_gb300")
    for dirpath, _, files in os.walk(pkg):
        for f in files:
            if f.endswith((".py", ".cu", ".cuh", ".h")):
                src = open(os.path.join(dirpath, f)).read()
                assert not re.search(r"^\s*(import|from)\s+oracle\b", src, re.M), f
                assert "tinylu_oracle" not in src, f


RANK_SCRIPT = r"""
import os, sys
sys.path.insert(0, sys.argv[1])
import torch.distributed as dist
import bench
dist.init_process_group("gloo", init_method="tcp://127.0.0.1:" + sys.argv[2],
                        rank=int(sys.argv[3]), world_size=2)
r = dist.get_rank()
seed = bench.rank_seed(1236, r)
t = bench.max_over_ranks(10.0 + 5.0 * r, dist)
print(f"rank={r} seed={seed} max={t}")
dist.barrier()
dist.destroy_process_group()
"""


def test_two_rank_logic_on_gloo(tmp_path):
    pytest.importorskip("torch.distributed")
    script = tmp_path / "ranks.py"
    script.write_text(RANK_SCRIPT)
    import socket
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = str(s.getsockname()[1])
    s.close()
    procs = [subprocess.Popen([sys.executable, str(script), ROOT, port, str(r)], stdout=subprocess.PIPE,
                              stderr=subprocess.PIPE, text=True) for r in range(2)]
    outs = [p.communicate(timeout=120) for p in procs]
    for p, (o, e) in zip(procs, outs):
        assert p.returncode == 0, e
    lines = sorted(o.strip() for o, _ in outs)
    assert lines[0] == "rank=0 seed=1236 max=15.0"
    assert lines[1] == "rank=1 seed=1336 max=15.0"
