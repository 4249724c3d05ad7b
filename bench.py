#!/usr/bin/env python3
"""Benchmark of the batched FP64 LUpp hot path on GB300.

One step = the standalone FP64 sweep (every n in 1..32, 2^20 systems per n
capped at 6 GiB of A, b, x, ipiv and info per n; half U[-1,1] entries, half
A = U diag(s) V^T with kappa log-uniform in [1e2, 1e8]; b = A x_true), all
systems resident in HBM in the interleaved batch-minor layout, solved by
tl_gesv_batched.  The per-system layout sweep is timed the same way and
reported beside it; when the fused Newton kernel is available the Norton
integration over 2^22 points is timed too.

Prints ONE JSON line (rank 0).  `--impl reference` times the CPU oracle on a
bounded sample of the same workload instead (the reference arm).
"""
import argparse
import json
import math
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

import numpy as np  # noqa: E402

METRIC = "FP64 tiny-LUpp solves/s vs n; Newton points/s; p50/p99 request latency"
UNIT = "solves/s"
CAP_BYTES = 6 * (1 << 30)
SWEEP_BATCH = 1 << 20
NEWTON_POINTS = 1 << 22


_T0 = time.perf_counter()


def rank_seed(base, rank):
    """Per-rank seed: every rank solves its own independent batch (weak
    scaling, no data exchanged)."""
    return base + 100 * rank


def max_over_ranks(value, dist, device=None):
    """Step time of the job = the slowest rank's (max over ranks)."""
    if dist is None or not dist.is_initialized():
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def log(msg):
    sys.stderr.write(f"[bench {time.perf_counter() - _T0:8.1f}s] {msg}\n")
    sys.stderr.flush()


def sweep_batch(n, full=SWEEP_BATCH):
    """2^20 systems, capped so A, b, x, ipiv and info fit in 6 GiB."""
    per = 8 * n * n + 16 * n + 4 * n + 4
    return min(full, CAP_BYTES // per)


def flops_per_system(n):
    """Algorithmic FP64 flops of one fused getrf + getrs (FMA = 2 flops):
    getrf (n-1)n(2n-1)/6 FMAs, n(n-1)/2 multipliers, n-1 reciprocals;
    getrs n(n-1) FMAs and n divisions."""
    fma = (n - 1) * n * (2 * n - 1) // 6 + n * (n - 1)
    return 2 * fma + n * (n - 1) // 2 + (n - 1) + n


def bytes_per_system(n):
    """A and b read, x, ipiv (int32) and info (int32) written."""
    return 8 * n * n + 8 * n + 8 * n + 4 * n + 4


# FP64 pipe of the GB300 from its unit counts: 152 SMs x 4 sub-partitions x
# 0.5 DFMA lane/clock (one warp-wide DFMA per 64 clocks per sub-partition) x
# 2 flops x 2.07 GHz maximum SM clock.  The roofline denominator is the rate
# tl_measure_fma_peak measures in the same run; this figure is reported
# beside it.
FP64_PEAK_DERIVED_TFLOPS = 152 * 4 * 0.5 * 2 * 2.07e9 / 1e12


# DRAM bytes per system measured by ncu for the current kernels, keyed by
# (variant, n): dram__bytes_read.sum + dram__bytes_write.sum of one launch
# (ncu flushes the caches before it) / systems in the launch.  An entry must
# be removed whenever its kernel changes.
DRAM_BYTES_PER_SYSTEM = {(116, 30): 7747, (116, 29): 7257, (116, 28): 6773, (132, 32): 8783, (208, 23): 4684,
                         (208, 22): 4300}

VARIANT_NAMES = {1: "k_factor_thread", 2: "k_factor_group<T=2>", 4: "k_factor_group<T=4>",
                 8: "k_factor_group<T=8>", 16: "k_factor_group<T=16>",
                 102: "k_smem_group<T=2, lane tile>", 104: "k_smem_group<T=4, lane tile>",
                 108: "k_smem_group<T=8, lane tile>", 116: "k_smem_group<T=16, element walk>",
                 132: "k_smem_group<T=32, element walk>", 202: "k_smem_group<T=2, element walk>",
                 204: "k_smem_group<T=4, element walk>", 208: "k_smem_group<T=8, element walk>"}


def load_peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        with open(p) as f:
            return json.load(f)
    except OSError:
        return {}


class Clocks:
    """Samples SM clock and throttle reasons with nvidia-smi during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None

    def __enter__(self):
        try:
            self.proc = subprocess.Popen(["nvidia-smi", "-i", str(self.index), f"--query-gpu={self.Q}",
                                          "--format=csv,noheader,nounits", "-lms", "200"],
                                         stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
        return self

    def __exit__(self, *exc):
        self.lines = []
        if self.proc is not None:
            self.proc.terminate()
            try:
                out, _ = self.proc.communicate(timeout=5)
            except subprocess.TimeoutExpired:
                self.proc.kill()
                out, _ = self.proc.communicate()
            self.lines = [ln for ln in out.splitlines() if ln.strip()]

    def summary(self):
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in getattr(self, "lines", []):
            f = [x.strip() for x in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for nm, v in zip(names, f[5:9]):
                if v.lower() == "active":
                    reasons.add(nm)
        if not sm:
            return None
        top = max(sm)
        loaded = [v for v in sm if v >= 0.5 * top] or sm
        return {"sm_mhz": statistics.median(loaded), "sm_max_mhz": mx, "reasons": sorted(reasons),
                "samples": len(sm)}


# ---------------------------------------------------------------------------
# workload
# ---------------------------------------------------------------------------

def make_sweep(n_list, layout, seed_base, device, torch, L, I, cap=None):
    """Generate every n's batch on the device and pack it in `layout`."""
    data = {}
    for n in n_list:
        S = sweep_batch(n) if cap is None else min(cap, sweep_batch(n))
        log(f"generate n={n} batch={S} layout={layout}")
        A, b, _x = I.sweep_systems_torch(n, S, seed_base * 1000 + n, device)
        ld = L.pad_ld(S)
        dA = L.matrices_to_layout(A, layout, ld)
        db = L.vectors_to_layout(b, layout, ld)
        del A, b, _x
        rows = n * (ld if layout == 1 else S)
        data[n] = dict(S=S, ld=ld, A=dA, b=db, x=torch.empty(rows, dtype=torch.float64, device=device),
                       ipiv=torch.empty(rows, dtype=torch.int32, device=device),
                       info=torch.empty(S, dtype=torch.int32, device=device))
    torch.cuda.synchronize()
    return data


def run_sweep(tl, h, data, layout, stream, torch, events=None):
    for n, d in data.items():
        if events is not None:
            events[n][0].record(stream)
        st = tl.tl_gesv_batched(h, n, d["A"], None, d["b"], d["x"], d["ipiv"], d["info"], layout, d["ld"],
                                d["S"], stream.cuda_stream)
        if st != 0:
            tl.check("tl_gesv_batched", st, h)
        if events is not None:
            events[n][1].record(stream)


def time_sweep(tl, h, data, layout, steps, warmup, torch, dist_barrier):
    stream = torch.cuda.current_stream()
    for _ in range(warmup):
        run_sweep(tl, h, data, layout, stream, torch)
    torch.cuda.synchronize()
    per_n = {n: [] for n in data}
    dist_barrier()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    ev = {n: (torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)) for n in data}
    step_ms = []
    for _ in range(steps):
        t0.record(stream)
        run_sweep(tl, h, data, layout, stream, torch, ev)
        t1.record(stream)
        t1.synchronize()
        step_ms.append(t0.elapsed_time(t1))
        for n in data:
            per_n[n].append(ev[n][0].elapsed_time(ev[n][1]))
    torch.cuda.synchronize()
    dist_barrier()
    return step_ms, per_n


def host_link_gbs(torch, device, nbytes=1 << 32, reps=3):
    """Pinned host <-> device copy bandwidth of this machine (GB/s, best of
    `reps` copies of `nbytes` each way), the reference the end-to-end rate
    is read against."""
    hbuf = torch.empty(nbytes, dtype=torch.uint8).pin_memory()
    dbuf = torch.empty(nbytes, dtype=torch.uint8, device=device)
    out = {}
    for name, (dst, src) in (("h2d", (dbuf, hbuf)), ("d2h", (hbuf, dbuf))):
        best = 1e30
        for _ in range(reps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record()
            dst.copy_(src, non_blocking=True)
            e1.record()
            e1.synchronize()
            best = min(best, e0.elapsed_time(e1))
        out[name] = nbytes / (best / 1e3) / 1e9
    del hbuf, dbuf
    return out


def sweep_e2e(tl, h, n_list, layout, steps, warmup, torch, device, L, I, seed):
    """Same sweep through host buffers: every step copies each n's A and b
    from pinned host memory, solves, and copies x, ipiv and info back.  One
    pinned pool backs every n's inputs: the sweep recipe's batch of the
    largest n (half U[-1,1], half kappa-controlled), in the layout; smaller n
    read its leading entries.  The copies and solves are pipelined over the
    sizes: copy-in, solve and copy-out run on their own streams with two
    device buffer sets, so the next size's inputs cross the link while the
    current size solves."""
    sizes = {}
    h2d = d2h = 0
    for n in n_list:
        S = sweep_batch(n)
        ld = L.pad_ld(S)
        rows = n * (ld if layout == 1 else S)
        sizes[n] = (S, ld, n * rows, rows)
        h2d += (n * rows + rows) * 8
        d2h += rows * 8 + rows * 4 + S * 4
    bigA = max(v[2] for v in sizes.values())
    bigv = max(v[3] for v in sizes.values())
    bigS = max(v[0] for v in sizes.values())
    n_pool = max(n_list, key=lambda n: sizes[n][2])
    S, ld = sizes[n_pool][0], sizes[n_pool][1]
    A, b, _x = I.sweep_systems_torch(n_pool, S, seed, device)
    hA = torch.empty(bigA, dtype=torch.float64).pin_memory()
    hb = torch.empty(bigv, dtype=torch.float64).pin_memory()
    hA[:sizes[n_pool][2]].copy_(L.matrices_to_layout(A, layout, ld).reshape(-1)[:sizes[n_pool][2]])
    hb[:sizes[n_pool][3]].copy_(L.vectors_to_layout(b, layout, ld).reshape(-1)[:sizes[n_pool][3]])
    del A, b, _x
    torch.cuda.empty_cache()
    hx = [torch.empty(bigv, dtype=torch.float64).pin_memory() for _ in range(2)]
    hp = [torch.empty(bigv, dtype=torch.int32).pin_memory() for _ in range(2)]
    hi = [torch.empty(bigS, dtype=torch.int32).pin_memory() for _ in range(2)]
    dA = [torch.empty(bigA, dtype=torch.float64, device=device) for _ in range(2)]
    db = [torch.empty(bigv, dtype=torch.float64, device=device) for _ in range(2)]
    dx = [torch.empty(bigv, dtype=torch.float64, device=device) for _ in range(2)]
    dp = [torch.empty(bigv, dtype=torch.int32, device=device) for _ in range(2)]
    di = [torch.empty(bigS, dtype=torch.int32, device=device) for _ in range(2)]
    main = torch.cuda.current_stream()
    s_in, s_sol, s_out = (torch.cuda.Stream() for _ in range(3))

    def one_step():
        start = torch.cuda.Event()
        start.record(main)
        for s_ in (s_in, s_sol, s_out):
            s_.wait_event(start)
        freed = [None, None]
        for idx, n in enumerate(n_list):
            S, ld, na, nv = sizes[n]
            k = idx % 2
            if freed[k] is not None:
                s_in.wait_event(freed[k])      # buffer k's previous results are home
            with torch.cuda.stream(s_in):
                dA[k][:na].copy_(hA[:na], non_blocking=True)
                db[k][:nv].copy_(hb[:nv], non_blocking=True)
            loaded = torch.cuda.Event()
            loaded.record(s_in)
            s_sol.wait_event(loaded)
            st = tl.tl_gesv_batched(h, n, dA[k], None, db[k], dx[k], dp[k], di[k], layout, ld, S,
                                    s_sol.cuda_stream)
            if st != 0:
                tl.check("tl_gesv_batched", st, h)
            solved = torch.cuda.Event()
            solved.record(s_sol)
            s_out.wait_event(solved)
            with torch.cuda.stream(s_out):
                hx[k][:nv].copy_(dx[k][:nv], non_blocking=True)
                hp[k][:nv].copy_(dp[k][:nv], non_blocking=True)
                hi[k][:S].copy_(di[k][:S], non_blocking=True)
            freed[k] = torch.cuda.Event()
            freed[k].record(s_out)
        for s_ in (s_in, s_sol, s_out):
            end = torch.cuda.Event()
            end.record(s_)
            main.wait_event(end)

    for _ in range(warmup):
        one_step()
    torch.cuda.synchronize()
    t0 = torch.cuda.Event(enable_timing=True)
    t1 = torch.cuda.Event(enable_timing=True)
    ms = []
    for _ in range(steps):
        t0.record(main)
        one_step()
        t1.record(main)
        t1.synchronize()
        ms.append(t0.elapsed_time(t1))
    total = sum(v[0] for v in sizes.values())
    med = statistics.median(ms)
    link = host_link_gbs(torch, device)
    return {"value": total / (med / 1e3), "unit": UNIT, "h2d_bytes_per_step": h2d, "d2h_bytes_per_step": d2h,
            "ms_per_step": med, "h2d_gb_per_s": h2d / (med / 1e3) / 1e9,
            "host_link_gb_per_s": link, "h2d_frac_of_link": h2d / (med / 1e3) / 1e9 / link["h2d"],
            "inputs": f"one pinned host pool: the sweep batch of n={n_pool} (half U[-1,1], half kappa in [1e2,1e8], "
                      "b = A x_true) in the layout, whose leading entries back every n's A and b; copy-in, solve "
                      "and copy-out pipelined over the sizes on three streams"}


# FP64 flops of one Norton law evaluation with its Jacobian and the residual
# norm: every operation on a value that depends on the point's data, counted
# on the oracle's code (sqrt and division count 1, parameter-only products
# excluded): strain trace 2, stress 18, mean stress 3, deviator 3, s:s 12,
# seq 2, flow direction 12, powers 4, residual 20, Jacobian 153 (c 2,
# 36 x (n_i n_j, 1.5K - nn, c*v, +delta) 144, g 1, last row 6), norm 15.
NORTON_EVAL_FLOPS = 244
NORTON_LU_FLOPS = flops_per_system(7)


def newton_bench(tl, h, steps, warmup, torch, device, I, seed, peak, npoints=NEWTON_POINTS, cpu_driven_steps=3):
    """Norton Newton over npoints (n = 7): the fused per-point kernel
    (Algorithm 2) in points/s with its FP64 fraction, and the batched,
    CPU-driven loop (Algorithm 1) on the same points beside it."""
    sig0, deps = I.norton_points_torch(npoints, seed, device)
    fields = torch.cat([sig0.t(), deps.t()], dim=0).contiguous()  # (12, npoints)
    del sig0, deps
    x = torch.empty((7, npoints), dtype=torch.float64, device=device)
    sig = torch.empty((6, npoints), dtype=torch.float64, device=device)
    it = torch.empty(npoints, dtype=torch.int32, device=device)
    st = torch.empty(npoints, dtype=torch.int32, device=device)
    law = tl.make_law(tl.TL_LAW_NORTON, 7, (200000.0, 0.3, 1e-12, 4.0, 1.0))
    stream = torch.cuda.current_stream()

    def timed(entry, name, k, w):
        def run():
            r = entry(h, law, npoints, fields, x, sig, it, st, 1e-10, 20, stream.cuda_stream)
            if r != 0:
                tl.check(name, r, h)
        for _ in range(w):
            run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(k):
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    med = timed(tl.tl_newton_integrate, "tl_newton_integrate", steps, warmup)
    iters = it.to(torch.int64)
    total_it = int(iters.sum().item())
    flops = total_it * NORTON_LU_FLOPS + (total_it + npoints) * NORTON_EVAL_FLOPS
    status = torch.bincount(st.to(torch.int64), minlength=4).tolist()
    out = {"points": npoints, "ms": med, "points_per_s": npoints / (med / 1e3),
           "mean_iterations": total_it / npoints, "max_iterations": int(iters.max().item()),
           "status_counts": status[:4], "fp64_tflops": flops / (med / 1e3) / 1e12,
           "fp64_frac": flops / (med / 1e3) / 1e12 / peak,
           "flops_model": "per solve 300 (LU n=7) + per law evaluation 244"}
    if cpu_driven_steps > 0:
        x_f, it_f, st_f = x.clone(), it.clone(), st.clone()
        med_cd = timed(tl.tl_newton_integrate_cpu_driven, "tl_newton_integrate_cpu_driven", cpu_driven_steps, 1)
        same = bool(torch.equal(it, it_f) and torch.equal(st, st_f) and
                    torch.equal(x.view(torch.int64), x_f.view(torch.int64)))
        out["cpu_driven"] = {"ms": med_cd, "points_per_s": npoints / (med_cd / 1e3),
                             "fused_speedup": med_cd / med, "iterations": int(iters.max().item()) + 1,
                             "results_equal_fused": same,
                             "launches_per_iteration": "assemble + gesv (+ fixup) + update, D2H count"}
        del x_f, it_f, st_f
    return out


def tanh_newton_bench(tl, h, steps, warmup, torch, device, I, seed, peak, npoints=1 << 17, sizes=(7, 13, 20, 32)):
    """The tanh law of the served stream, one size class at a time: the
    fused kernel's points/s, linear solves/s and the FP64 fraction of the
    solves alone (flops(n) per solve; the law's assembly is not counted)."""
    out = {}
    stream = torch.cuda.current_stream()
    for n in sizes:
        fields = I.tanh_points_torch(n, npoints, seed + n, device)
        x = torch.empty((n, npoints), dtype=torch.float64, device=device)
        it = torch.empty(npoints, dtype=torch.int32, device=device)
        st = torch.empty(npoints, dtype=torch.int32, device=device)
        law = tl.make_law(tl.TL_LAW_TANH, n)

        def run():
            r = tl.tl_newton_integrate(h, law, npoints, fields, x, None, it, st, 1e-10, 20, stream.cuda_stream)
            if r != 0:
                tl.check("tl_newton_integrate", r, h)
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        ms = []
        for _ in range(steps):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        med = statistics.median(ms)
        solves = int(it.to(torch.int64).sum().item())
        out[n] = {"points": npoints, "ms": med, "points_per_s": npoints / (med / 1e3),
                  "mean_iterations": solves / npoints, "solves_per_s": solves / (med / 1e3),
                  "lu_fp64_frac": solves * flops_per_system(n) / (med / 1e3) / 1e12 / peak,
                  "converged": int((st == 0).sum().item())}
        del fields, x, it, st
        torch.cuda.empty_cache()
    return out


# ---------------------------------------------------------------------------
# ragged batch, binary64 vs binary32 factor + binary64 refinement
# ---------------------------------------------------------------------------

RAGGED_N = (6, 7, 12, 13, 19, 25, 32)
RAGGED_W = (0.2, 0.25, 0.15, 0.15, 0.1, 0.1, 0.05)
RAGGED_BATCH = 1 << 20


def make_ragged_torch(batch, seed, device, torch, I):
    """2^20 systems with n drawn from RAGGED_N (weights RAGGED_W); each n's
    systems follow the sweep recipe (half U[-1,1], half kappa in [1e2,1e8],
    b = A x_true), stored per system column-major one after another in
    system order (so sizes are mixed in memory)."""
    g = torch.Generator(device=device)
    g.manual_seed(seed)
    w = torch.tensor(RAGGED_W, dtype=torch.float64, device=device)
    pick = torch.multinomial(w, batch, replacement=True, generator=g)
    sizes = torch.tensor(RAGGED_N, dtype=torch.int64, device=device)[pick]
    nn2 = sizes * sizes
    a_off = torch.cumsum(nn2, 0) - nn2
    b_off = torch.cumsum(sizes, 0) - sizes
    Abuf = torch.empty(int(nn2.sum().item()), dtype=torch.float64, device=device)
    bbuf = torch.empty(int(sizes.sum().item()), dtype=torch.float64, device=device)
    xtrue = torch.empty_like(bbuf)
    buckets = {}
    for n in RAGGED_N:
        idx = torch.nonzero(sizes == n).flatten()
        if idx.numel() == 0:
            continue
        A, b, x = I.sweep_systems_torch(n, idx.numel(), seed * 1000 + n, device)
        ia = (a_off[idx][:, None] + torch.arange(n * n, device=device)[None, :]).flatten()
        ib = (b_off[idx][:, None] + torch.arange(n, device=device)[None, :]).flatten()
        Abuf[ia] = A.transpose(1, 2).reshape(-1)
        bbuf[ib] = b.reshape(-1)
        xtrue[ib] = x.reshape(-1)
        buckets[n] = (idx, ia, ib)
        del A, b, x
    return dict(sizes=sizes.to(torch.int32), a_off=a_off, b_off=b_off, A=Abuf, b=bbuf, xtrue=xtrue,
                buckets=buckets, batch=batch)


def ragged_errors(d, x, torch):
    """Worst normwise backward error (in units of n * eps) and forward error
    against x_true (relative, inf-norm) over all systems solved (info 0)."""
    eps = 2.0 ** -52
    be_max, fe_max = 0.0, 0.0
    for n, (idx, ia, ib) in d["buckets"].items():
        A = d["A"][ia].reshape(-1, n, n).transpose(1, 2)
        xs = x[ib].reshape(-1, n)
        r = d["b"][ib].reshape(-1, n) - torch.matmul(A, xs[:, :, None])[:, :, 0]
        den = A.abs().sum(dim=2).amax(dim=1) * xs.abs().amax(dim=1) * eps * n
        ok = torch.isfinite(xs).all(dim=1)
        be = (r.abs().amax(dim=1) / den)[ok]
        xt = d["xtrue"][ib].reshape(-1, n)
        fe = ((xs - xt).abs().amax(dim=1) / xt.abs().amax(dim=1))[ok]
        be_max = max(be_max, float(be.max().item()) if be.numel() else 0.0)
        fe_max = max(fe_max, float(fe.max().item()) if fe.numel() else 0.0)
    return be_max, fe_max


def ragged_bench(tl, h, steps, warmup, torch, device, I, seed, batch=RAGGED_BATCH):
    """One tl_lupp_solve_batched call over the mixed-size batch, binary64
    and binary32-factor + binary64-refinement, each timed on its own."""
    d = make_ragged_torch(batch, seed, device, torch, I)
    x = torch.empty_like(d["b"])
    ipiv = torch.empty(d["b"].numel(), dtype=torch.int32, device=device)
    info = torch.empty(batch, dtype=torch.int32, device=device)
    ref = torch.empty(batch, dtype=torch.int32, device=device)
    stream = torch.cuda.current_stream()
    out = {"workload": "2^20 systems, n in {6,7,12,13,19,25,32} with weights {.2,.25,.15,.15,.1,.1,.05}, "
                       "half U[-1,1], half kappa in [1e2,1e8], b = A x_true; per-system column-major, sizes "
                       "mixed in memory; one tl_lupp_solve_batched call",
           "bytes_A": d["A"].numel() * 8}

    def timed(run):
        for _ in range(warmup):
            run()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        ms = []
        for _ in range(steps):
            e0.record(stream)
            run()
            e1.record(stream)
            e1.synchronize()
            ms.append(e0.elapsed_time(e1))
        return statistics.median(ms)

    legs = (("fp64", tl.TL_PREC_FP64, tl.TL_RAGGED_PERSISTENT),
            ("fp64_per_size_launches", tl.TL_PREC_FP64, tl.TL_RAGGED_PER_SIZE),
            ("fp32_ir", tl.TL_PREC_FP32_IR, tl.TL_RAGGED_PERSISTENT))
    piv_ref = None
    for name, prec, mode in legs:
        def run():
            st = tl.tl_lupp_solve_batched(h, batch, d["sizes"], d["a_off"], d["A"], d["b_off"], d["b"], x,
                                          d["b_off"], ipiv, info, prec, ref if prec else None,
                                          stream.cuda_stream)
            if st != 0:
                tl.check("tl_lupp_solve_batched", st, h)
        tl.check("tl_ragged_set_mode", tl.tl_ragged_set_mode(h, mode), h)
        med = timed(run)
        tl.tl_ragged_set_mode(h, tl.TL_RAGGED_PERSISTENT)
        be, fe = ragged_errors(d, x, torch)
        out[name] = {"ms": med, "solves_per_s": batch / (med / 1e3), "max_backward_error_n_eps": be,
                     "max_forward_error_vs_x_true": fe,
                     "info_nonzero": int((info != 0).sum().item()),
                     "launches": "bucketing (3) + plan + 1 persistent" if mode == tl.TL_RAGGED_PERSISTENT
                                 else "bucketing (3) + 32 per-size"}
        if prec:
            hist = torch.bincount((ref + 1).to(torch.int64), minlength=5).tolist()
            out[name]["refine_steps_hist"] = {"fallback": hist[0], "0": hist[1], "1": hist[2], "2": hist[3],
                                              "3": hist[4]}
        elif piv_ref is None:
            piv_ref = ipiv.clone()
        else:
            out[name]["pivots_equal_persistent"] = bool(torch.equal(ipiv, piv_ref))
    # the same systems as homogeneous per-n batches (bucketed and copied into
    # contiguous per-system arrays outside the timed region), one
    # tl_gesv_batched launch per size with the tuned per-n kernels
    per_n = {}
    for n, (idx, ia, ib) in d["buckets"].items():
        S = idx.numel()
        per_n[n] = dict(S=S, A=d["A"][ia].contiguous(), b=d["b"][ib].contiguous(),
                        x=torch.empty(S * n, dtype=torch.float64, device=device),
                        p=torch.empty(S * n, dtype=torch.int32, device=device),
                        i=torch.empty(S, dtype=torch.int32, device=device))

    def run_plain():
        for n, q in per_n.items():
            st = tl.tl_gesv_batched(h, n, q["A"], None, q["b"], q["x"], q["p"], q["i"], 0, q["S"], q["S"],
                                    stream.cuda_stream)
            if st != 0:
                tl.check("tl_gesv_batched", st, h)
    med = timed(run_plain)
    same = all(torch.equal(q["p"], piv_ref[d["buckets"][n][2]]) for n, q in per_n.items())
    out["fp64_plain_per_n_gesv"] = {"ms": med, "solves_per_s": batch / (med / 1e3),
                                    "launches": f"{len(per_n)} tl_gesv_batched (+ fixup passes)",
                                    "pivots_equal_persistent": same,
                                    "inputs": "pre-bucketed contiguous per-n copies (bucketing not timed)"}

    # the same launches fed from the mixed layout: the gather of each size's
    # A and b into contiguous per-n arrays (index_select, known indices) is
    # part of the timed region, as a caller holding a mixed batch would pay
    def run_gather_plain():
        for n, (idx, ia, ib) in d["buckets"].items():
            q = per_n[n]
            torch.index_select(d["A"], 0, ia, out=q["A"])
            torch.index_select(d["b"], 0, ib, out=q["b"])
        run_plain()
    med_g = timed(run_gather_plain)
    out["fp64_plain_per_n_gesv_with_gather"] = {"ms": med_g, "solves_per_s": batch / (med_g / 1e3),
                                                "launches": f"{2 * len(per_n)} gathers + {len(per_n)} tl_gesv_batched"}
    out["persistent_vs_plain_per_n"] = out["fp64_plain_per_n_gesv"]["ms"] / out["fp64"]["ms"]
    out["persistent_vs_plain_per_n_with_gather"] = med_g / out["fp64"]["ms"]
    out["persistent_vs_per_size_launches"] = out["fp64_per_size_launches"]["ms"] / out["fp64"]["ms"]
    out["fp32_ir_speedup"] = out["fp64"]["ms"] / out["fp32_ir"]["ms"]
    del d, per_n
    return out


# ---------------------------------------------------------------------------
# served Newton stream (continuous batching vs plain per-request launches)
# ---------------------------------------------------------------------------

SERVE_TANH_N = (7, 13, 20, 32)
SERVE_MAX_PTS = 1 << 16
SERVE_BUDGET = 20 * (1 << 30)


class ServeWorkload:
    """Request classes of the served stream: 30% Norton n = 7 points (the
    Newton workload), 70% tanh-law points with n uniform in {7, 13, 20, 32}
    (A = nI + U[-1,1], c in U[0.5,2], b in U[-3,3] n); request sizes
    log-uniform in [1k, 64k] points.  Inputs come from one page-locked pool
    per class (requests read its first `count` points through ld_in);
    outputs go to a ring of page-locked output slots."""

    def __init__(self, tl, torch, I, seed, out_slots=96):
        self.tl = tl
        g = np.random.default_rng(seed)
        self.pools = {}
        P = SERVE_MAX_PTS
        sig0, deps = I.norton_points(P, seed)
        f = np.concatenate([sig0.T, deps.T], axis=0)
        self.pools["norton"] = torch.from_numpy(np.ascontiguousarray(f)).pin_memory()
        for n in SERVE_TANH_N:
            A, c, b = I.tanh_points(n, P, seed + n)
            f = np.concatenate([A.transpose(0, 2, 1).reshape(P, n * n).T, c.T, b.T], axis=0)
            self.pools[n] = torch.from_numpy(np.ascontiguousarray(f)).pin_memory()
            del A, c, b, f
        self.laws = {"norton": tl.make_law(tl.TL_LAW_NORTON, 7, (200000.0, 0.3, 1e-12, 4.0, 1.0))}
        for n in SERVE_TANH_N:
            self.laws[n] = tl.make_law(tl.TL_LAW_TANH, n)
        self.out = [dict(x=torch.empty(32 * P, dtype=torch.float64).pin_memory(),
                         it=torch.empty(P, dtype=torch.int32).pin_memory(),
                         st=torch.empty(P, dtype=torch.int32).pin_memory()) for _ in range(out_slots)]
        self.g = g

    def draw(self, count):
        """count request descriptors: (class, points)."""
        out = []
        for _ in range(count):
            cls = "norton" if self.g.random() < 0.3 else int(self.g.choice(SERVE_TANH_N))
            pts = int(np.exp(self.g.uniform(np.log(1000), np.log(SERVE_MAX_PTS))))
            out.append((cls, pts))
        return out

    def request(self, cls, pts, slot):
        tl = self.tl
        o = self.out[slot]
        return tl.make_request(tl.TL_REQ_NEWTON, pts, self.pools[cls].data_ptr(), o["x"].data_ptr(),
                               o["it"].data_ptr(), o["st"].data_ptr(), law=self.laws[cls], ld_in=SERVE_MAX_PTS)


def run_stream(tl, h, wl, reqs, arrivals, mode):
    """Submit reqs[i] at arrivals[i] seconds (None: all at once) to a server
    in `mode` and wait for all.  Returns latencies, makespan and lags."""
    cap, slots = (1 << 18, 4) if mode == "batched" else (0, 1)
    st, srv = tl.tl_server_create(h, SERVE_BUDGET, slots, cap, 1e-10, 20)
    tl.check("tl_server_create", st, h)
    free_slots = list(range(len(wl.out)))
    inflight = {}   # id -> (slot, descriptor, submission delay after the arrival)
    lat, lag = [], []
    t0 = time.perf_counter()

    def reap(block=False):
        for rid in list(inflight):
            if block:
                s2, rs, l = tl.tl_server_wait(srv, rid, 600.0)
                done = 1
            else:
                s2, done, rs, l = tl.tl_server_test(srv, rid)
            if s2 == 0 and done:
                if rs != 0:
                    raise RuntimeError(f"request failed: {rs}")
                slot, _, delay = inflight.pop(rid)
                lat.append(l + delay)     # latency counted from the arrival
                free_slots.append(slot)

    for i, (cls, pts) in enumerate(reqs):
        due = t0 + (arrivals[i] if arrivals is not None else 0.0)
        if arrivals is not None:
            while True:
                now = time.perf_counter()
                if now >= due:
                    break
                if due - now > 0.0005:
                    reap()
                    time.sleep(min(0.0005, due - now - 0.0003))
        while not free_slots:
            reap()
        slot = free_slots.pop()
        req = wl.request(cls, pts, slot)
        delay = max(0.0, time.perf_counter() - due) if arrivals is not None else 0.0
        lag.append(delay)
        s2, rid = tl.tl_server_submit(srv, req)
        tl.check("tl_server_submit", s2, h)
        inflight[rid] = (slot, req, delay)
    reap(block=True)
    makespan = time.perf_counter() - t0
    _, stats = tl.tl_server_stats_get(srv)
    tl.tl_server_destroy(srv)
    return lat, makespan, lag, stats


def serve_bench(tl, h, torch, I, seed, burst=160, seconds=3.0):
    wl = ServeWorkload(tl, torch, I, seed)
    out = {"workload": "served Newton stream: 30% Norton n=7, 70% tanh law n in {7,13,20,32}; request sizes "
                       "log-uniform in [1k, 64k] points; Poisson arrivals; host page-locked inputs and outputs "
                       "(H2D and D2H inside every request's latency); 20 GiB device arena",
           "batched": {"slots": 4, "max_points_per_tick": 1 << 18}, "plain": {"slots": 1, "one_request_per_tick": True}}
    # capacity: a burst of requests submitted at once
    reqs = wl.draw(burst)
    pts = sum(p for _, p in reqs)
    for mode in ("batched", "plain"):
        run_stream(tl, h, wl, reqs[:8], None, mode)   # warm-up
        # the burst three times; the run of median makespan is reported
        runs = sorted((run_stream(tl, h, wl, reqs, None, mode) for _ in range(3)), key=lambda r: r[1])
        lat, span, _, stats = runs[1]
        out[mode]["capacity_points_per_s"] = pts / span
        out[mode]["capacity_requests_per_s"] = burst / span
        out[mode]["capacity_points_per_s_runs"] = [pts / r[1] for r in runs]
        out[mode]["ticks_in_burst"] = stats["ticks"]
        # where the burst's time went: the union of the server's kernel
        # intervals (CUDA events) and the request loop's host time per tick
        out[mode]["device_busy_fraction"] = stats["kernel_busy_s"] / span
        out[mode]["host_enqueue_ms_per_tick"] = stats["host_enqueue_s"] / max(1, stats["ticks"]) * 1e3
    cap_rps = out["batched"]["capacity_requests_per_s"]
    mean_pts = pts / burst
    for load in (0.5, 0.8, 0.95):
        rate = load * cap_rps
        count = max(50, int(rate * seconds))
        reqs = wl.draw(count)
        arrivals = np.cumsum(wl.g.exponential(1.0 / rate, size=count))
        for mode in ("batched", "plain"):
            lat, span, lag, stats = run_stream(tl, h, wl, reqs, arrivals, mode)
            lat_ms = np.array(lat) * 1e3
            out[mode][f"load_{int(load * 100)}"] = {
                "offered_requests_per_s": rate, "requests": count,
                "points_per_s": sum(p for _, p in reqs) / span,
                "p50_ms": float(np.percentile(lat_ms, 50)), "p99_ms": float(np.percentile(lat_ms, 99)),
                "max_ms": float(lat_ms.max()), "ticks": stats["ticks"],
                "submit_lag_p99_ms": float(np.percentile(np.array(lag) * 1e3, 99))}
    out["mean_points_per_request"] = mean_pts
    del wl
    return out


# ---------------------------------------------------------------------------
# CPU oracle timing (cpu_baseline and the reference arm)
# ---------------------------------------------------------------------------

def oracle_sweep_rate(n_list, target_s=0.3, samples=None, seed_base=1236, max_sample=1 << 15):
    """Time the oracle on a bounded sample of each n's batch and extrapolate
    to the full sweep.  Returns (solves/s over the sweep, threads, sample)."""
    import oracle
    from paper_2609_15217_gb300 import inputs as I
    threads = oracle.max_threads()
    total_S = 0
    total_t = 0.0
    sample = {}
    for n in n_list:
        m = samples[n] if samples else 256
        A, b, _, _ = I.sweep_systems(n, m, seed_base * 1000 + n)
        t = time.perf_counter()
        oracle.gesv(A, b)
        dt = time.perf_counter() - t
        if not samples:
            m2 = int(min(sweep_batch(n), max_sample, max(256, m * target_s / max(dt, 1e-6))))
            A, b, _, _ = I.sweep_systems(n, m2, seed_base * 1000 + n)
            t = time.perf_counter()
            oracle.gesv(A, b)
            dt = time.perf_counter() - t
            m = m2
        sample[n] = m
        S = sweep_batch(n)
        total_S += S
        total_t += S * dt / m
    return total_S / total_t, threads, sample


def sweep_config(n_list, world, systems=None):
    """The `config` object of the contract line (both arms)."""
    return {"workload": "standalone FP64 sweep: n=1..32, 2^20 systems per n capped at 6 GiB "
                        "(n>=27), half U[-1,1], half kappa in [1e2,1e8], b=A x_true; interleaved "
                        "batch-minor layout, tl_gesv_batched",
            "systems_per_step": systems if systems is not None else sum(sweep_batch(n) for n in n_list),
            "L2": "inputs larger than L2 (each step streams "
                  f"{sum(bytes_per_system(n) * sweep_batch(n) for n in n_list) / 1e9:.1f} GB)",
            "parallelism": f"replicas x{world}"}


def reference_arm(args):
    """--impl reference: the CPU oracle (as it stands) on the host cores."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    n_list = list(range(args.nmin, args.nmax + 1))
    vals = []
    sample = None
    t_all = time.perf_counter()
    for i in range(args.warmup + args.steps):
        v, threads, sample = oracle_sweep_rate(n_list, target_s=args.ref_seconds_per_n, samples=sample)
        if i >= args.warmup:
            vals.append(v)
    v = statistics.median(vals)
    sample_desc = ("oracle gesv on the first m_n systems of each n's sweep batch (m_n per n: "
                   + ", ".join(f"{n}:{m}" for n, m in sample.items())
                   + "), time extrapolated linearly to the full per-n batch sizes")
    out = {
        "impl": "reference", "metric": METRIC, "value": v, "unit": UNIT, "n_gpus": args.gpus,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": sum(sweep_batch(n) for n in n_list) / v * 1e3, "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": sweep_config(n_list, 1),
        "cpu_baseline": {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle", "sample": sample_desc},
        "e2e": {"value": v, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
        "wall_s": time.perf_counter() - t_all,
    }
    print(json.dumps(out))


# ---------------------------------------------------------------------------

def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=5)
    ap.add_argument("--warmup", type=int, default=3)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--nmin", type=int, default=1)
    ap.add_argument("--nmax", type=int, default=32)
    ap.add_argument("--no-per-system", action="store_true")
    ap.add_argument("--no-e2e", action="store_true")
    ap.add_argument("--no-cpu", action="store_true")
    ap.add_argument("--no-newton", action="store_true")
    ap.add_argument("--no-ragged", action="store_true")
    ap.add_argument("--no-serve", action="store_true")
    ap.add_argument("--no-autotune", action="store_true")
    ap.add_argument("--variant", type=int, default=None,
                    help="force one kernel variant (lanes + 100 * storage) for every n of the sweep")
    ap.add_argument("--dispatch-table", default=None,
                    help="interleaved-layout dispatch table (JSON written by tl_autotune) to apply instead of "
                         "autotuning, e.g. to profile the same kernels the timed run used")
    ap.add_argument("--batch", type=int, default=None,
                    help="cap on systems per n (small cases for profiling; the default is the full sweep)")
    ap.add_argument("--ref-seconds-per-n", type=float, default=0.3)
    args = ap.parse_args()
    if args.impl == "reference":
        return reference_arm(args)

    import torch
    from paper_2609_15217_gb300 import inputs as I
    from paper_2609_15217_gb300 import layout as L
    from paper_2609_15217_gb300 import tinylu as tl

    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    dist = None
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
    device = torch.device("cuda", local)
    torch.cuda.set_device(device)

    def barrier():
        if dist is not None:
            dist.barrier()

    h = tl.tl_create()
    n_list = list(range(args.nmin, args.nmax + 1))
    tune = {}
    if args.variant is not None:
        for n in range(args.nmin, args.nmax + 1):
            tl.check("tl_dispatch_set", tl.tl_dispatch_set(h, n, 1, args.variant, 0), h)
        tune[1] = {n: args.variant for n in range(args.nmin, args.nmax + 1)}
    elif args.dispatch_table:
        with open(args.dispatch_table) as f:
            entries = json.load(f)["entries"]
        for e in entries:
            tl.check("tl_dispatch_set", tl.tl_dispatch_set(h, e["n"], 1, e["variant"], e["block"]), h)
        tune[1] = {e["n"]: e["variant"] for e in entries}
    elif not args.no_autotune:
        # size-aware dispatcher: time every kernel variant per n once, before
        # anything is timed (the "best X" selection of the paper's Sec. 4.1)
        log("autotune")
        for layout in (1, 0):
            path = os.path.join(ROOT, f"_build/autotune_layout{layout}.json")
            os.makedirs(os.path.dirname(path), exist_ok=True)
            tl.check("tl_autotune", tl.tl_autotune(h, args.nmin, args.nmax, layout, path), h)
            with open(path) as f:
                tune[layout] = {e["n"]: e["variant"] for e in json.load(f)["entries"]}
    if not args.no_autotune and not args.no_ragged:
        # lanes per system of the persistent ragged launch and the
        # mixed-precision route, per n
        log("autotune ragged")
        path = os.path.join(ROOT, "_build/autotune_ragged.json")
        tl.check("tl_autotune_ragged", tl.tl_autotune_ragged(h, 1, 32, path), h)
        with open(path) as f:
            tune["ragged"] = {e["n"]: {"lanes": e["lanes"], "mixed_refines": e["mixed_refines"],
                                       "ir_variant": e["ir_variant"],
                                       "ms_fp64": round(e["ms_fp64"], 4), "ms_mixed": round(e["ms_mixed"], 4)}
                              for e in json.load(f)["entries"]}
    t_gen = time.perf_counter()
    data = make_sweep(n_list, 1, rank_seed(1236, rank), device, torch, L, I, args.batch)
    gen_s = time.perf_counter() - t_gen

    # FP64 pipe rate of this GPU, measured before and after the timed sweep
    # (independent DFMA chains on every SM); the faster is the roofline peak
    peaks = []

    def measure_peak():
        st, tf, per_clk, mhz = tl.tl_measure_fma_peak(h, 64)
        tl.check("tl_measure_fma_peak", st, h)
        peaks.append({"tflops": tf, "dfma_lanes_per_clk_per_sm": per_clk, "sm_mhz": mhz})

    measure_peak()
    log("timing interleaved sweep")
    with Clocks(local) as clk:
        step_ms, per_n = time_sweep(tl, h, data, 1, args.steps, args.warmup, torch, barrier)
    clocks = clk.summary()
    measure_peak()
    peak = max(p["tflops"] for p in peaks)
    st32, fp32_tf, fp32_clk, _ = tl.tl_measure_fma_peak(h, 32)
    tl.check("tl_measure_fma_peak", st32, h)

    med_step = max_over_ranks(statistics.median(step_ms), dist, device)
    systems_rank = sum(d["S"] for d in data.values())
    value = systems_rank * world / (med_step / 1e3)

    per_n_out = {}
    flops_total = 0.0
    for n, d in data.items():
        ms = statistics.median(per_n[n])
        f = flops_per_system(n) * d["S"]
        flops_total += f
        per_n_out[n] = {"batch": d["S"], "ms": round(ms, 4), "solves_per_s": d["S"] / (ms / 1e3),
                        "fp64_tflops": f / (ms / 1e3) / 1e12,
                        "fp64_frac": f / (ms / 1e3) / 1e12 / peak,
                        "gbs": bytes_per_system(n) * d["S"] / (ms / 1e3) / 1e9}
    # dominant kernel: the variant (thread-to-system mapping + storage) with
    # the largest share of the step; its largest launch is the roofline unit
    variant_of = {n: tl.tl_dispatch_get(h, n, 1)[1] for n in per_n_out}
    fam_ms = {}
    for n, v in variant_of.items():
        fam_ms[v] = fam_ms.get(v, 0.0) + per_n_out[n]["ms"]
    fam = max(fam_ms, key=fam_ms.get)
    fam_n = sorted(n for n in per_n_out if variant_of[n] == fam)
    dom = max(fam_n, key=lambda n: per_n_out[n]["ms"])
    dom_flops = flops_per_system(dom) * data[dom]["S"]
    achieved = dom_flops / (per_n_out[dom]["ms"] / 1e3) / 1e12
    fam_flops = sum(flops_per_system(n) * data[n]["S"] for n in fam_n)
    traffic = DRAM_BYTES_PER_SYSTEM.get((fam, dom))
    roofline = {"bound": "alu", "pipe": "fp64",
                "kernel": f"{VARIANT_NAMES.get(fam, fam)} (variant {fam}), gesv n={dom} interleaved launch",
                "achieved": achieved, "peak": peak, "unit": "TFLOP/s",
                "frac": achieved / peak,
                "traffic": traffic * data[dom]["S"] if traffic else None,
                "traffic_source": "ncu dram__bytes_read.sum + dram__bytes_write.sum per system on a smaller batch "
                                  "of the same kernel and n, scaled to the launch" if traffic else
                                  "null: no ncu DRAM counters taken on the current version of this kernel",
                "peak_source": "measured in this run by tl_measure_fma_peak (independent DFMA chains, 4 x 256 "
                               "threads per SM, CUDA events), faster of the probes before and after the sweep",
                "peak_probes": peaks,
                "peak_derived": FP64_PEAK_DERIVED_TFLOPS,
                "peak_derived_source": "152 SMs x 4 SMSPs x 0.5 DFMA/clk x 2 flop x 2.07 GHz",
                "fp32_fma_peak_tflops": fp32_tf, "fp32_ffma_lanes_per_clk_per_sm": fp32_clk,
                "kernel_share_of_step": fam_ms[fam] / sum(fam_ms.values()),
                "kernel_n": fam_n,
                "kernel_fp64_frac": fam_flops / (fam_ms[fam] / 1e3) / 1e12 / peak,
                "sweep_fp64_frac": flops_total / (med_step / 1e3) / 1e12 / peak,
                # the per-n evidence for ">= 0.60 of the FP64 roofline for n >= 8"
                "per_n_fp64_frac": [round(per_n_out[n]["fp64_frac"], 3) for n in sorted(per_n_out)],
                "per_n_variant": [variant_of[n] for n in sorted(per_n_out)],
                "per_n_first": min(per_n_out)}
    del data
    torch.cuda.empty_cache()

    extra = {}
    if not args.no_per_system:
        log("per-system layout sweep")
        data_ps = make_sweep(n_list, 0, rank_seed(1236, rank), device, torch, L, I, args.batch)
        ms_ps, per_n_ps = time_sweep(tl, h, data_ps, 0, max(2, args.steps // 2), 1, torch, barrier)
        sys_ps = sum(d["S"] for d in data_ps.values())
        extra["per_system_layout"] = {
            "value": sys_ps * world / (statistics.median(ms_ps) / 1e3), "unit": UNIT,
            "ms_per_step": statistics.median(ms_ps),
            "per_n_solves_per_s": {n: data_ps[n]["S"] / (statistics.median(per_n_ps[n]) / 1e3) for n in data_ps}}
        del data_ps
        torch.cuda.empty_cache()

    if not args.no_newton:
        log("newton")
        extra["newton"] = newton_bench(tl, h, max(2, args.steps // 2), 2, torch, device, I, rank_seed(1237, rank),
                                       peak)
        extra["newton"]["points_per_s"] *= world
        torch.cuda.empty_cache()
        log("newton tanh")
        extra["newton_tanh"] = tanh_newton_bench(tl, h, max(2, args.steps // 2), 2, torch, device, I,
                                                 rank_seed(1239, rank), peak)
        for v in extra["newton_tanh"].values():
            v["points_per_s"] *= world
            v["solves_per_s"] *= world

    if not args.no_ragged:
        log("ragged batch, binary64 and mixed precision")
        extra["ragged"] = ragged_bench(tl, h, max(2, args.steps // 2), 2, torch, device, I, rank_seed(1238, rank))
        for k in ("fp64", "fp32_ir"):
            extra["ragged"][k]["solves_per_s"] *= world
        torch.cuda.empty_cache()

    if not args.no_serve and world == 1:
        log("served Newton stream")
        extra["serve"] = serve_bench(tl, h, torch, I, rank_seed(1239, rank))
        torch.cuda.empty_cache()

    e2e = None
    if not args.no_e2e:
        log("end-to-end sweep")
        e2e = sweep_e2e(tl, h, n_list, 1, max(2, args.steps // 2), 1, torch, device, L, I,
                        rank_seed(1240, rank) * 1000 + args.nmax)
        e2e["value"] *= world
        torch.cuda.empty_cache()

    cpu = None
    if rank == 0 and world == 1 and not args.no_cpu:
        log("cpu baseline")
        v, threads, sample = oracle_sweep_rate(n_list)
        cpu = {"value": v, "unit": UNIT, "cores": threads, "kind": "oracle",
               "sample": "oracle gesv (OpenMP over systems) on the first m_n systems of each n's sweep batch "
                         f"({sum(sample.values())} systems in total, ~0.3 s per n), extrapolated to the full "
                         "per-n batch sizes"}

    log("done")
    # one launch per n and step, plus the fixup launch that follows the
    # one-thread register kernels (variant 1) on the same stream
    launches = sum(2 if tl.tl_dispatch_get(h, n, 1)[1] == 1 else 1 for n in n_list) * args.steps
    tl.tl_destroy(h)
    if rank == 0:
        out = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world, "steps": args.steps,
            "warmup": args.warmup, "ms_per_step": med_step, "higher_is_better": True, "scaling": "weak",
            "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "config": sweep_config(n_list, world, systems_rank),
            "roofline": roofline, "cpu_baseline": cpu, "e2e": e2e, "gpu_launches": launches,
            "clocks": clocks, "per_n": per_n_out, "gen_s": gen_s, "dispatch": tune, **extra,
        }
        print(json.dumps(out))
    if dist is not None:
        dist.destroy_process_group()


if __name__ == "__main__":
    main()
