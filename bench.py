#!/usr/bin/env python
"""Benchmark of exact sparse products over Z/mZ on one GB300 (or N replicas).

Workload (one step): y = A*x and z = A^T*x (mod m) on the 1M x 1M power-law
matrix (Zipf row lengths, mean 16, max 10 000, ~15.8M nonzeros, uniform
distinct columns), m = 65521, through the library's plan.  Inputs are
resident in HBM; L2 is flushed (a 256 MB write) between timed steps, outside
the timed events.  Throughput is Gnnz*vec/s: nonzeros times vectors per
second (the paper's Mflops / 2000).

Also printed, in the same JSON line:
  roofline      achieved algorithmic GB/s of the A*x kernel vs measured HBM peak
  e2e           the same step with x on pinned host memory and y, z copied back
  cpu_baseline  the CPU oracle on this host (bounded sample)
  clocks        SM clocks sampled during the timed region
  extra         other formats and moduli, the block Wiedemann sequence
                (persistent kernel vs one launch per kernel), the batched launch,
                products over GF(2) with bit-packed vectors, and the
                polynomial-matrix product of the sigma-basis step

  python bench.py [--gpus N] [--steps K] [--warmup W] [--impl reference]
"""
from __future__ import annotations

import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import threading
import time

import numpy as np

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

import gen  # noqa: E402

METRIC = "mod-p SpMV Gnnz*vec/s"
UNIT = "Gnnz*vec/s"
WORKLOAD = ("powerlaw 1M x 1M, Zipf row lengths mean 16 max 10k (15.8M nnz), m=65521; "
            "step = y=A*x and z=A^T*x")
SEED = 1002
FALLBACK_HBM = 6800.0
NOMINAL_HBM = 7900.0   # GB/s, GB300's nominal HBM3e bandwidth (context beside the measured peak)


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--modulus", type=int, default=65521)
    ap.add_argument("--format", default="AUTO")
    ap.add_argument("--extras", default="formats,multivec,batch,sequence,sigma,gf2,polymat",
                    help="comma list from formats,multivec,batch,sequence,sigma,gf2,polymat "
                         "('' for none)")
    ap.add_argument("--cpu-seconds", type=float, default=8.0,
                    help="seconds of oracle work for each of the single-thread and all-core "
                         "CPU baselines")
    ap.add_argument("--profile", default="",
                    help="'ax' or 'atx': only run warm-up + --steps launches of that product; "
                         "'seq': one block sequence of --steps steps on the 100k Wiedemann "
                         "matrix; 'polymat': three 16 x 16 polynomial-matrix products of degree "
                         "6250; 'sigma': one sigma-basis of [S(x); -I] for a uniform 16 x 16 "
                         "sequence of --steps terms (no timing, no extras), for an ncu capture")
    return ap.parse_args()


def peaks():
    p = os.path.join(ROOT, "MEASURED_PEAKS.json")
    try:
        d = json.load(open(p))
        return float(d["hbm_gbs"]), "measured"
    except Exception:
        return FALLBACK_HBM, "fallback"


class Clocks:
    """nvidia-smi samples of SM clock and throttle reasons during a region."""

    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.proc = None
        self.lines = []

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.index}", f"--query-gpu={self.Q}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
            self.t = threading.Thread(target=self._read, daemon=True)
            self.t.start()
        except Exception:
            self.proc = None

    def _read(self):
        for line in self.proc.stdout:
            self.lines.append(line.strip())

    def wait_first(self, timeout=3.0):
        """Block until the sampler has printed its first sample (its start-up
        queries are then over), at most `timeout` seconds."""
        t0 = time.time()
        while self.proc and not self.lines and time.time() - t0 < timeout:
            time.sleep(0.01)

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["nvidia-smi unavailable"]}
        time.sleep(0.25)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, mx, reasons = [], None, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for ln in self.lines:
            f = [t.strip() for t in ln.split(",")]
            if len(f) < 9:
                continue
            try:
                sm.append(float(f[1]))
                mx = float(f[2])
            except ValueError:
                continue
            for n, v in zip(names, f[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        return {"sm_mhz": statistics.median(sm) if sm else None, "sm_max_mhz": mx,
                "reasons": sorted(reasons), "samples": len(sm)}


def algorithmic_bytes(A, m):
    """Sec. 2.1 CSR traffic of one y = A*x with the +-1 entries value-free
    (Sec. 2.4.2): per nonzero a 4-byte column index, plus a value (2 bytes if
    m <= 2^16, 4 otherwise) unless the entry is +1 or -1 (value 1 or m - 1),
    plus 4(n+1) bytes of row pointers, 4n of x and 4n of y."""
    vb = 2 if m <= 65536 else 4
    v = np.asarray(A.val, dtype=np.uint64) % m
    general = int(A.nnz - np.count_nonzero((v == 1) | (v == m - 1)))
    return 4 * A.nnz + vb * general + 4 * (A.nrows + 1) + 4 * A.ncols + 4 * A.nrows


def traffic_record(kernel_key):
    """DRAM bytes per launch from the committed ncu summary, if it was taken
    on the current kernel sources (else None)."""
    p = os.path.join(ROOT, "profiles", "traffic.json")
    try:
        d = json.load(open(p))
    except Exception:
        return None
    rec = d.get(kernel_key)
    if not rec or rec.get("source_hash") != kernel_source_hash():
        return None
    return rec.get("dram_bytes_per_launch")


def kernel_source_hash():
    h = hashlib.sha256()
    for f in ("kernels.cu", "plan.cu", "panel.cu", "ff_internal.cuh"):
        h.update(open(os.path.join(ROOT, "paper_1004_3719_gb300", "csrc", f), "rb").read())
    return h.hexdigest()[:16]


def host_cores():
    try:
        return len(os.sched_getaffinity(0))
    except Exception:
        return os.cpu_count() or 1


def oracle_steps(A, x, seconds, threads):
    """The oracle's y = A x and z = A^T x on this host, repeated for about
    `seconds` (at least once) on `threads` host threads (rows split
    statically); returns (steps, seconds)."""
    import oracle
    n = 0
    t0 = time.perf_counter()
    while True:
        oracle.csr_spmv(A, x, threads=threads)
        oracle.csr_spmv_transpose(A, x, threads=threads)
        n += 1
        if time.perf_counter() - t0 >= seconds:
            break
    return n, time.perf_counter() - t0


def cpu_baseline(A, x, seconds):
    """The oracle on all host cores (the reported baseline) and on one."""
    cores = host_cores()
    n1, t1 = oracle_steps(A, x, seconds, 1)
    nc, tc = oracle_steps(A, x, seconds, cores)
    return {"value": round(2 * A.nnz * nc / tc / 1e9, 4), "unit": UNIT, "cores": cores,
            "kind": "oracle",
            "sample": f"{nc} steps (y=A*x, z=A^T*x) on the full matrix, rows split over "
                      f"{cores} threads, {tc:.1f} s",
            "single_thread": {"value": round(2 * A.nnz * n1 / t1 / 1e9, 4), "cores": 1,
                              "sample": f"{n1} steps, one thread, {t1:.1f} s"}}


def shard(count, rank, world):
    """The units of `rank` when `count` independent units (problems, replicas)
    are split over `world` ranks, round robin; no data moves between ranks."""
    return list(range(rank, count, world))


def max_over_ranks(dist, value, device="cpu"):
    """Largest `value` over all ranks (the job's time is its slowest rank's)."""
    if dist is None:
        return value
    import torch
    t = torch.tensor([float(value)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def dist_setup(args):
    world = int(os.environ.get("WORLD_SIZE", "1"))
    rank = int(os.environ.get("RANK", "0"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pg = None
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl" if args.impl == "ours" else "gloo")
        pg = dist
    return world, rank, local, pg


def run_reference(args):
    world, rank, local, pg = dist_setup(args)
    if rank != 0:
        return
    import oracle
    oracle.build()
    A = gen.powerlaw_matrix(seed=SEED, m=args.modulus)
    x = gen.uniform_block(SEED, A.ncols, 1, args.modulus)
    cores = host_cores()
    for _ in range(args.warmup):
        oracle.csr_spmv(A, x, threads=cores)
        oracle.csr_spmv_transpose(A, x, threads=cores)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.csr_spmv(A, x, threads=cores)
        oracle.csr_spmv_transpose(A, x, threads=cores)
    dt = time.perf_counter() - t0
    val = 2 * A.nnz * args.steps / dt / 1e9
    print(json.dumps({
        "impl": "reference", "metric": METRIC, "value": round(val, 4), "unit": UNIT,
        "n_gpus": args.gpus, "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(dt / args.steps * 1e3, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "modulus": args.modulus},
        "cpu_baseline": {"value": round(val, 4), "unit": UNIT, "cores": cores, "kind": "oracle",
                         "sample": f"{args.steps} timed steps of the full workload, rows split "
                                   f"over {cores} threads"},
        "e2e": {"value": round(val, 4), "unit": UNIT, "h2d_bytes_per_step": 0,
                "d2h_bytes_per_step": 0}}))


class L2Flush:
    """Evict L2 between timed steps: write a 256 MB buffer (twice the L2),
    then read another one, so that the lines left in L2 are clean and no
    write-back of the flush lands inside the next timed step."""

    def __init__(self, torch):
        self.w = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")
        self.r = torch.zeros(64 << 20, dtype=torch.int32, device="cuda")

    def fill_(self, v=1):
        self.w.fill_(v)
        self.sink = self.r.sum()


def timed_steps(torch, fn, steps, flush, stream):
    """Sum of per-step device times (ms), L2 flushed before every step."""
    evs = []
    for _ in range(steps):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        fn()
        e1.record(stream)
        evs.append((e0, e1))
    torch.cuda.synchronize()
    return [a.elapsed_time(b) for a, b in evs]


def warm_times(torch, ff, M, x, y, z, stream, reps=50):
    """Warm figures beside the L2-flushed ones: `reps` back-to-back y = A x
    (then z = A^T x) with no flush between them, one pair of events around
    each run of `reps`; the matrix (about 100 MB per direction) partly stays
    in the 129 MB L2 from one product to the next."""
    sp = stream.cuda_stream
    out = {"reps": reps, "l2": "not flushed between products"}
    for key, fn, o in (("ax", ff.spmv_apply, y), ("atx", ff.spmv_apply_transpose, z)):
        for _ in range(3):
            fn(M.handle, x, 1, o, 1, 1, 1, 0, sp)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(reps):
            fn(M.handle, x, 1, o, 1, 1, 1, 0, sp)
        e1.record(stream)
        torch.cuda.synchronize()
        us = e0.elapsed_time(e1) * 1e3 / reps
        out[key] = {"us": round(us, 2), "gnnz_s": round(M.info()["nnz"] / us / 1e3, 1)}
    return out


def extra_formats(torch, ff, flush, stream, moduli=(65521, 2**31 - 1, 3)):
    sp = stream.cuda_stream
    out = {}
    fmts = ["AUTO", "CSR", "ELLR", "COO", "COOS", "DIA", "HYBRID", "BINNED", "PANEL", "LEARNED", "EXHAUSTIVE"]
    sel_of = {"LEARNED": ff.SEL.LEARNED, "EXHAUSTIVE": ff.SEL.EXHAUSTIVE}
    for m in moduli:
        A = gen.powerlaw_matrix(seed=SEED, m=m)
        x = torch.from_numpy(gen.uniform_block(SEED, A.ncols, 1, m).view(np.int32)).cuda()
        y = torch.empty(A.nrows, dtype=torch.int32, device="cuda")
        row = {}
        for f in fmts:
            for pm in ((0, 1) if m == 3 else (-1,)):
                key = f if pm < 0 else f"{f}{'+pm1' if pm else '-nopm1'}"
                try:
                    if f in sel_of:
                        # FMT.AUTO under that selector: it picks the layout
                        # (x-panel or binned) and the per-bin formats
                        M = ff.Matrix.from_csr(A, selector=sel_of[f], priority_format=ff.FMT.AUTO,
                                               transpose_mode=ff.TRANSPOSE.NONE, use_pm1=pm)
                    else:
                        M = ff.Matrix.from_csr(A, priority_format=getattr(ff.FMT, f),
                                               transpose_mode=ff.TRANSPOSE.NONE, use_pm1=pm)
                except ff.FFSPMVError as e:
                    row[key] = f"n/a ({e.status == 5 and 'size guard' or e})"
                    continue
                fn = lambda: ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, sp)
                for _ in range(3):
                    fn()
                t = timed_steps(torch, fn, 10, flush, stream)
                ms = statistics.median(t)
                row[key] = {"gnnz_s": round(A.nnz / ms / 1e6, 1),
                            "gbs": round(algorithmic_bytes(A, m) / ms / 1e6, 1),
                            "ms": round(ms, 4)}
                if f in sel_of or f == "AUTO":
                    row[key]["layout"] = "panel" if "panels" in M.describe() else "binned"
                del M
        out[f"m={m}"] = row
    return out


def extra_multivec(torch, ff, flush, stream):
    """Y = A X on the 1M power-law matrix (m = 65521) for blocks of 1 to 16
    vectors through AUTO (the x-panel layout): passes of 4 or 2 vectors read
    the matrix once for all of them (Sec. 2.5.1), next to the time of that
    many single-vector products."""
    sp = stream.cuda_stream
    m = 65521
    A = gen.powerlaw_matrix(seed=SEED, m=m)
    M = ff.Matrix.from_csr(A, transpose_mode=ff.TRANSPOSE.NONE)
    res = {"workload": f"powerlaw 1M x 1M ({A.nnz} nnz), m={m}, AUTO, L2 flushed"}
    single = None
    for nv in (1, 2, 4, 8, 16):
        x = torch.from_numpy(gen.uniform_block(SEED, A.ncols, nv, m).view(np.int32)).cuda()
        y = torch.empty((A.nrows, nv), dtype=torch.int32, device="cuda")
        fn = lambda: ff.spmv_apply(M.handle, x, nv, y, nv, nv, 1, 0, sp)
        for _ in range(3):
            fn()
        ms = statistics.median(timed_steps(torch, fn, 10, flush, stream))
        single = ms if nv == 1 else single
        res[f"nvec={nv}"] = {"ms": round(ms, 4), "gnnz_vec_s": round(A.nnz * nv / ms / 1e6, 1),
                             "launches": M.launches(False, nv),
                             "vs_nvec_single_products": round(nv * single / ms, 2)}
    return res


def extra_sequence(torch, ff, stream):
    sp = stream.cuda_stream
    p, s = 65521, 16
    W = gen.wiedemann_matrix(seed=1003)
    n = W.nrows
    L = 2 * n // s + 2
    X = torch.from_numpy(gen.uniform_block(1003, n, s, p).view(np.int32)).cuda()
    Y = torch.from_numpy(gen.uniform_block(1003, n, s, p, key=1).view(np.int32)).cuda()
    res = {"workload": f"wiedemann 100k x 100k ({W.nnz} nnz), s=16, p=65521, {L} steps"}
    for mode, name in ((0, "persistent_graph"), (1, "per_launch")):
        M = ff.Matrix.from_csr(W, sequence_mode=mode, transpose_mode=ff.TRANSPOSE.NONE)
        S = torch.empty((L, s, s), dtype=torch.int32, device="cuda")
        ff.spmv_block_sequence(M.handle, X, Y, s, 0, L, S, None, sp)
        torch.cuda.synchronize()
        ts = []
        for _ in range(3 if mode == 0 else 1):
            e0 = torch.cuda.Event(enable_timing=True)
            e1 = torch.cuda.Event(enable_timing=True)
            e0.record(stream)
            ff.spmv_block_sequence(M.handle, X, Y, s, 0, L, S, None, sp)
            e1.record(stream)
            torch.cuda.synchronize()
            ts.append(e0.elapsed_time(e1))
        ms = min(ts)
        res[name] = {"ms": round(ms, 3), "us_per_step": round(ms * 1e3 / L, 3),
                     "gnnz_vec_s": round(W.nnz * s * (L - 1) / ms / 1e6, 1)}
        del M
    return res


def extra_sigma(torch, ff, stream):
    """The sigma-basis step of block Wiedemann on the 100k workload: the
    12 502-term sequence S_i = X^T A^i Y (s = 16) from the GPU, then the
    order-12 502 sigma-basis of [S(x); -I] (32 x 16), synchronous call."""
    sp = stream.cuda_stream
    p, s = 65521, 16
    W = gen.wiedemann_matrix(seed=1003)
    n = W.nrows
    L = 2 * n // s + 2
    X = torch.from_numpy(gen.uniform_block(1003, n, s, p).view(np.int32)).cuda()
    Y = torch.from_numpy(gen.uniform_block(1003, n, s, p, key=1).view(np.int32)).cuda()
    M = ff.Matrix.from_csr(W, transpose_mode=ff.TRANSPOSE.NONE)
    S = M.block_sequence(X, Y, L, stream=sp)
    F = ff.sigma_wiedemann_input(p, S, stream=sp)
    torch.cuda.synchronize()
    ts = []
    for _ in range(2):
        t0 = time.perf_counter()
        _, delta, deg = ff.sigma_basis(p, F, stream=sp)
        torch.cuda.synchronize()
        ts.append((time.perf_counter() - t0) * 1e3)
    rows = sorted(range(2 * s), key=lambda i: (delta[i], i))[:s]
    return {"workload": f"sigma-basis of [S(x); -I], 32 x 16, order {L}, p={p} (100k Wiedemann sequence)",
            "ms": round(min(ts), 1), "generator_row_degree_sum": sum(delta[i] for i in rows),
            "basis_degree_bound": deg,
            "degrees_sum_to_s_L": sum(delta) == s * L}  # det P = c x^(s L) for [S; -I]


def extra_batch(torch, ff, stream):
    sp = stream.cuda_stream
    probs = gen.batch_problems(seed=1004)
    mats = [ff.Matrix.from_csr(A, transpose_mode=ff.TRANSPOSE.NONE, priority_format=ff.FMT.CSR)
            for A, _ in probs]
    xs = [torch.from_numpy(np.ascontiguousarray(
        gen.uniform_block(7 + j, A.ncols, s, A.modulus)).view(np.int32)).cuda()
        for j, (A, s) in enumerate(probs)]
    ys = [torch.empty((A.nrows, s) if s > 1 else (A.nrows,), dtype=torch.int32, device="cuda")
          for A, s in probs]
    nv = [s for _, s in probs]
    work = sum(A.nnz * s for A, s in probs)

    def one_launch():
        ff.spmv_batch_apply([M.handle for M in mats], xs, ys, nv, sp)

    def per_matrix():
        for M, x, y, s in zip(mats, xs, ys, nv):
            ff.spmv_apply(M.handle, x, s, y, s, s, 1, 0, sp)

    res = {"workload": f"{len(probs)} matrices, {sum(A.nnz for A, _ in probs)} nnz, "
                       f"{work} nnz*vec per pass"}
    for name, fn in (("one_launch", one_launch), ("per_matrix_fixed_csr", per_matrix)):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        e0.record(stream)
        for _ in range(5):
            fn()
        e1.record(stream)
        torch.cuda.synchronize()
        ms = e0.elapsed_time(e1) / 5
        res[name] = {"ms": round(ms, 3), "gnnz_vec_s": round(work / ms / 1e6, 1)}
    return res


def extra_gf2(torch, ff, flush, stream):
    """Y = A X over GF(2) on the same power-law pattern (all values odd at
    m = 2), 64 and 256 vectors packed in 1 and 4 words per row."""
    sp = stream.cuda_stream
    A = gen.powerlaw_matrix(seed=SEED, m=2)
    M = ff.Matrix.from_csr(A, transpose_mode=ff.TRANSPOSE.NONE)
    hbm, _ = peaks()
    res = {"workload": f"powerlaw 1M x 1M pattern ({A.nnz} nnz), GF(2), L2 flushed"}
    for w in (1, 4):
        x = torch.from_numpy(gen.uniform_block(SEED, A.ncols, 2 * w, 2**32 - 1).view(np.int64)).cuda()
        y = torch.empty((A.nrows, w), dtype=torch.int64, device="cuda")
        fn = lambda: ff.spmv_apply_gf2(M.handle, 0, x, y, w, False, sp)
        for _ in range(3):
            fn()
        ms = statistics.median(timed_steps(torch, fn, 10, flush, stream))
        # algorithmic bytes: 4 per entry (column), 8 per row pointer, x and y words
        abytes = 4 * A.nnz + 8 * (A.nrows + 1) + 8 * w * (A.ncols + A.nrows)
        res[f"words={w}"] = {"ms": round(ms, 4), "gnnz_vec_s": round(A.nnz * 64 * w / ms / 1e6, 1),
                             "algorithmic_gbs": round(abytes / ms / 1e6, 1),
                             "hbm_frac": round(abytes / ms / 1e6 / hbm, 3)}
    return res


def extra_polymat(torch, ff, stream):
    """C = A B mod p for 16 x 16 polynomial matrices of degree 6250 each: the
    top-level product of PM-Basis on the block-Wiedemann sequence of the
    100k matrix (12 502 terms of 16 x 16)."""
    import ctypes
    sp = stream.cuda_stream
    p, s, d = 65521, 16, 6250
    A = torch.from_numpy(gen.uniform_block(21, (d + 1) * s, s, p).view(np.int32)).cuda().view(d + 1, s, s)
    B = torch.from_numpy(gen.uniform_block(22, (d + 1) * s, s, p).view(np.int32)).cuda().view(d + 1, s, s)
    C = torch.empty((2 * d + 1, s, s), dtype=torch.int32, device="cuda")
    need = ctypes.c_int64()
    L = ff.lib()
    L.polymat_mul_workspace(s, d, d, ctypes.byref(need))
    work = torch.empty(need.value, dtype=torch.uint8, device="cuda")
    fn = lambda: L.polymat_mul(p, s, d, d, A.data_ptr(), B.data_ptr(), C.data_ptr(), work.data_ptr(),
                               need.value, sp)
    for _ in range(3):
        fn()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(stream)
    for _ in range(10):
        fn()
    e1.record(stream)
    torch.cuda.synchronize()
    ms = e0.elapsed_time(e1) / 10
    schoolbook = s ** 3 * (d + 1) ** 2  # multiply-adds of the plain product
    return {"workload": f"{s}x{s} polynomial matrices, degree {d} each, p={p}, NTT length 16384 x 3 primes",
            "ms": round(ms, 3), "schoolbook_equivalent_gmac_s": round(schoolbook / ms / 1e6, 1)}


def main():
    args = parse()
    if args.impl == "reference":
        return run_reference(args)
    import torch
    world, rank, local, dist = dist_setup(args)
    torch.cuda.set_device(local)
    import paper_1004_3719_gb300 as ff
    ff.build()
    if args.profile == "polymat":
        p, s, d = 65521, 16, 6250
        A = gen.uniform_block(21, (d + 1) * s, s, p).reshape(d + 1, s, s)
        B = gen.uniform_block(22, (d + 1) * s, s, p).reshape(d + 1, s, s)
        for _ in range(3):
            ff.polymat_mul(p, A, B)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "polymat", "products": 3}))
        return
    if args.profile == "sigma":
        p, s = 65521, 16
        S = gen.uniform_block(23, args.steps * s, s, p).reshape(args.steps, s, s)
        _, delta, deg = ff.sigma_basis(p, ff.sigma_wiedemann_input(p, S))
        torch.cuda.synchronize()
        print(json.dumps({"profile": "sigma", "order": args.steps, "delta_sum": sum(delta), "degree_bound": deg}))
        return
    if args.profile == "seq":
        W = gen.wiedemann_matrix(seed=1003)
        X = torch.from_numpy(gen.uniform_block(1003, W.nrows, 16, 65521).view(np.int32)).cuda()
        Y = torch.from_numpy(gen.uniform_block(1003, W.nrows, 16, 65521, key=1).view(np.int32)).cuda()
        Mw = ff.Matrix.from_csr(W, transpose_mode=ff.TRANSPOSE.NONE)
        Mw.block_sequence(X, Y, args.steps)
        torch.cuda.synchronize()
        print(json.dumps({"profile": "seq", "steps": args.steps}))
        return
    m = args.modulus
    A = gen.powerlaw_matrix(seed=SEED, m=m)
    x_host = gen.uniform_block(SEED + rank, A.ncols, 1, m)
    M = ff.Matrix.from_csr(A, priority_format=getattr(ff.FMT, args.format))
    stream = torch.cuda.current_stream()
    sp = stream.cuda_stream
    x = torch.from_numpy(x_host.view(np.int32)).cuda()
    y = torch.empty(A.nrows, dtype=torch.int32, device="cuda")
    z = torch.empty(A.ncols, dtype=torch.int32, device="cuda")
    flush = L2Flush(torch)

    def step():
        ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, sp)
        ff.spmv_apply_transpose(M.handle, x, 1, z, 1, 1, 1, 0, sp)

    if args.profile:
        fn = ff.spmv_apply if args.profile == "ax" else ff.spmv_apply_transpose
        out = y if args.profile == "ax" else z
        for _ in range(args.warmup + args.steps):
            fn(M.handle, x, 1, out, 1, 1, 1, 0, sp)
        torch.cuda.synchronize()
        print(json.dumps({"profile": args.profile, "launches": M.launches(args.profile == "atx", 1),
                          "plan": M.describe().splitlines()[0]}))
        return

    # The clock sampler starts first; the warm-up steps (each like a timed
    # one: L2 flush, then the step) run once it is sampling, so that neither
    # its start-up nor the idle wait falls on the first timed step (measured:
    # a first step of 119 us against 37 us for the rest without this).
    clocks = Clocks(local)
    clocks.start()
    clocks.wait_first()
    time.sleep(0.1)
    for _ in range(max(args.warmup, 3)):
        flush.fill_(1)
        step()
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    torch.cuda.synchronize()
    evs = []
    for _ in range(args.steps):
        flush.fill_(1)
        e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
        e[0].record(stream)
        ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, sp)
        e[1].record(stream)
        ff.spmv_apply_transpose(M.handle, x, 1, z, 1, 1, 1, 0, sp)
        e[2].record(stream)
        evs.append(e)
    torch.cuda.synchronize()
    if dist:
        dist.barrier()
    clk = clocks.stop()
    t_step = [e[0].elapsed_time(e[2]) for e in evs]
    t_ax = [e[0].elapsed_time(e[1]) for e in evs]
    total_ms = max_over_ranks(dist, sum(t_step), "cuda")
    units = 2 * A.nnz * args.steps * world
    value = units / (total_ms / 1e3) / 1e9
    launches = args.steps * (M.launches(False, 1) + M.launches(True, 1))

    # end to end: x from pinned host memory, y and z back to pinned host memory
    xh = torch.from_numpy(x_host.view(np.int32)).pin_memory()
    yh = torch.empty(A.nrows, dtype=torch.int32).pin_memory()
    zh = torch.empty(A.ncols, dtype=torch.int32).pin_memory()
    # y goes back on a second stream while A^T*x runs; every copy is inside
    # the timed region (e1 waits for both streams)
    copy_stream = torch.cuda.Stream()
    e2e_ms = []
    for i in range(max(args.steps // 2, 5) + 2):
        flush.fill_(1)
        e0 = torch.cuda.Event(enable_timing=True)
        e1 = torch.cuda.Event(enable_timing=True)
        y_done, y_back = torch.cuda.Event(), torch.cuda.Event()
        e0.record(stream)
        x.copy_(xh, non_blocking=True)
        ff.spmv_apply(M.handle, x, 1, y, 1, 1, 1, 0, sp)
        y_done.record(stream)
        with torch.cuda.stream(copy_stream):
            copy_stream.wait_event(y_done)
            yh.copy_(y, non_blocking=True)
            y_back.record(copy_stream)
        ff.spmv_apply_transpose(M.handle, x, 1, z, 1, 1, 1, 0, sp)
        zh.copy_(z, non_blocking=True)
        stream.wait_event(y_back)
        e1.record(stream)
        torch.cuda.synchronize()
        if i >= 2:
            e2e_ms.append(e0.elapsed_time(e1))
    e2e_val = 2 * A.nnz / (statistics.mean(e2e_ms) / 1e3) / 1e9

    if rank != 0:
        return
    hbm, src = peaks()
    ax_ms = statistics.mean(t_ax)
    abytes = algorithmic_bytes(A, m)
    achieved = abytes / (ax_ms / 1e3) / 1e9
    fmt_a = M.describe().split(":")[0].split()[-1]
    kname = ("k_panel (y=A*x: one launch, x staged inside the kernel)" if fmt_a == "PANEL"
             else "k_plan (y=A*x)")
    roof = {"bound": "hbm", "achieved": round(achieved, 1), "peak": hbm, "unit": "GB/s",
            "frac": round(achieved / hbm, 4), "traffic": traffic_record(f"spmv_A_{m}_{fmt_a}"),
            "kernel": kname, "algorithmic_bytes": abytes,
            "peak_source": f"{src} (MEASURED_PEAKS.json hbm_gbs)" if src == "measured" else "fallback",
            "launch_ms": round(ax_ms, 4), "frac_of_nominal": round(achieved / NOMINAL_HBM, 4)}
    extra = {"plan": M.describe()}
    try:
        extra["warm"] = warm_times(torch, ff, M, x, y, z, stream)
    except Exception as e:  # report, do not hide
        extra["warm"] = f"failed: {type(e).__name__}: {e}"
    wanted = [e for e in args.extras.split(",") if e]
    del M
    torch.cuda.empty_cache()
    for name, fn in (("multivec", lambda: extra_multivec(torch, ff, flush, stream)),
                     ("polymat", lambda: extra_polymat(torch, ff, stream)),
                     ("gf2", lambda: extra_gf2(torch, ff, flush, stream)),
                     ("formats", lambda: extra_formats(torch, ff, flush, stream)),
                     ("sequence", lambda: extra_sequence(torch, ff, stream)),
                     ("sigma", lambda: extra_sigma(torch, ff, stream)),
                     ("batch", lambda: extra_batch(torch, ff, stream))):
        if name in wanted:
            try:
                extra[name] = fn()
            except Exception as e:  # report, do not hide
                extra[name] = f"failed: {type(e).__name__}: {e}"
    cpu = cpu_baseline(A, x_host, args.cpu_seconds) if world == 1 else None
    line = {
        "metric": METRIC, "value": round(value, 3), "unit": UNIT, "n_gpus": world,
        "steps": args.steps, "warmup": args.warmup,
        "ms_per_step": round(total_ms / args.steps, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "u32", "data": "synthetic",
        "config": {"workload": WORKLOAD, "format": args.format, "modulus": m,
                   "l2": "flushed (256 MB write) before every timed step, outside the events",
                   "parallelism": f"replicas x{world}" if world > 1 else "single GPU"},
        "roofline": roof, "cpu_baseline": cpu, "clocks": clk,
        "e2e": {"value": round(e2e_val, 3), "unit": UNIT,
                "h2d_bytes_per_step": 4 * A.ncols, "d2h_bytes_per_step": 4 * (A.nrows + A.ncols)},
        "gpu_launches": launches, "extra": extra,
    }
    print(json.dumps(line))


if __name__ == "__main__":
    main()
