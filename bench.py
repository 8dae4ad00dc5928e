"""Benchmark of the triangular solve L X = alpha B on one GB300 (or N replicas).

Default workload: the varlen batch of 8192 independent complex128 solves with
m, n uniform in [8, 64], alpha = (1.5, -0.5), non-unit diagonal, seed 0
(synthetic data from the seeded generator), one batched call per step.

    python bench.py [--gpus N] [--steps K] [--warmup W] [--impl ours|reference]
                    [--workload batched_c128|single_fp64_64|large_fp64|large_c128|mixed_r32|mixed_ir|serve]

Prints one JSON line.  Metric: GFLOP/s counted as m^2 n real flops per solve
(x4 for complex), whole job.  Under torchrun each rank solves its own batch
(seed offset by rank, "weak" scaling) with no collective on the data path.
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

METRIC = "TRSM GFLOP/s (m²n) and % roofline; mixed solves/s with p50/p99 latency"
# FP64 peak derived from the unit count: GB300's nominal 1.25 TFLOP/s FP64 is
# 2 FP64 FMA per clock per SM: 2 FMA x 2 flop x 152 SMs x 2070 MHz.
FP64_PEAK_GFLOPS = 2 * 2 * 152 * 2070e6 / 1e9
PEAKS_FILE = os.path.join(ROOT, "MEASURED_PEAKS.json")


def load_peaks():
    try:
        with open(PEAKS_FILE) as f:
            return json.load(f), "measured"
    except OSError:
        return {"hbm_gbs": 6800.0, "bf16_tflops": 1900.0, "bf16_tflops_sustained": 1700.0}, "fallback"


# ---------------------------------------------------------------------------
# distributed plumbing (timing only; no collective on the data path)
# ---------------------------------------------------------------------------
class Dist:
    def __init__(self):
        self.world = int(os.environ.get("WORLD_SIZE", "1"))
        self.rank = int(os.environ.get("RANK", "0"))
        self.local = int(os.environ.get("LOCAL_RANK", "0"))
        self.pg = None

    def init(self, backend):
        if self.world > 1:
            import torch.distributed as dist
            os.environ.setdefault("MASTER_ADDR", "127.0.0.1")
            dist.init_process_group(backend=backend)
            self.pg = dist

    def barrier(self):
        if self.pg is not None:
            self.pg.barrier()

    def max(self, x: float, device="cpu") -> float:
        if self.pg is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.MAX)
        return float(t.item())

    def sum(self, x: float, device="cpu") -> float:
        if self.pg is None:
            return x
        import torch
        t = torch.tensor([x], dtype=torch.float64, device=device)
        self.pg.all_reduce(t, op=self.pg.ReduceOp.SUM)
        return float(t.item())

    def close(self):
        if self.pg is not None:
            self.pg.destroy_process_group()


def shard_seed(base_seed: int, rank: int) -> int:
    """Each rank solves its own batch: the seed is offset by the rank."""
    return base_seed + 1000003 * rank


# ---------------------------------------------------------------------------
# clocks during the timed region
# ---------------------------------------------------------------------------
class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index: int):
        self.gpu = gpu_index
        self.samples = []
        self.proc = None
        self.window = None

    def start(self):
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu=timestamp,{self.FIELDS}", "--format=csv,noheader,nounits",
                 "-lms", "100"], stdout=subprocess.PIPE, stderr=subprocess.DEVNULL, text=True)
        except OSError:
            self.proc = None
            return
        self.thread = threading.Thread(target=self._read, daemon=True)
        self.thread.start()
        time.sleep(0.3)

    def _read(self):
        for line in self.proc.stdout:
            self.samples.append((time.time(), [x.strip() for x in line.split(",")]))

    def mark(self, t0, t1):
        self.window = (t0, t1)

    def stop(self):
        if self.proc is None:
            return None
        time.sleep(0.15)
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except subprocess.TimeoutExpired:
            self.proc.kill()
        rows = self.samples
        if self.window:
            inside = [r for (t, r) in rows if self.window[0] - 0.05 <= t <= self.window[1] + 0.05]
            rows = inside if inside else [r for (_, r) in rows]
        else:
            rows = [r for (_, r) in rows]
        sm, mx, reasons = [], 0.0, set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[2]))
                mx = max(mx, float(r[3]))
            except (ValueError, IndexError):
                continue
            for k, nm in enumerate(names):
                if len(r) > 6 + k and r[6 + k].lower().startswith("active"):
                    reasons.add(nm)
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": mx, "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------------------
# workloads
# ---------------------------------------------------------------------------
def source_sha(files):
    h = hashlib.sha256()
    for f in files:
        with open(os.path.join(ROOT, f), "rb") as fh:
            h.update(fh.read())
    return h.hexdigest()[:16]


def profile_traffic(name: str, files, work=None):
    """DRAM bytes per launch from a committed ncu summary, if it matches the current source.

    With `work` (algorithmic units of one launch of the bench's workload) and a
    summary that records `work_per_launch` for a smaller captured case, the
    captured bytes are scaled by work / work_per_launch."""
    path = os.path.join(ROOT, "profiles", name)
    try:
        kv = {}
        with open(path) as f:
            for line in f:
                if ":" in line:
                    k, v = line.split(":", 1)
                    kv[k.strip()] = v.strip()
        if kv.get("source_sha256_16") != source_sha(files):
            return None
        dram = float(kv["dram_bytes_per_launch"])
        if work is not None and "work_per_launch" in kv:
            return dram * work / float(kv["work_per_launch"])
        return dram
    except (OSError, KeyError, ValueError):
        return None


SMALL_SOURCES = ["paper_2608_25469_gb300/csrc/small.cu", "paper_2608_25469_gb300/csrc/common.cuh"]
PACKED_SOURCES = ["paper_2608_25469_gb300/csrc/packed.cu", "paper_2608_25469_gb300/csrc/common.cuh"]


def batched_inputs(seed, batch=8192, c64=False):
    """The config-1 batch (complex128; complex64 = the same values rounded)."""
    from paper_2608_25469_gb300 import inputs as I
    ms, ns = I.batched_sizes(seed, batch)
    As = [I.gen_A(seed, int(m), I.C128, inst=b) for b, m in enumerate(ms)]
    Bs = [I.gen_B(seed, int(m), int(n), I.C128, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    es = 16
    if c64:
        As = [np.asfortranarray(a.astype(np.complex64)) for a in As]
        Bs = [np.asfortranarray(b.astype(np.complex64)) for b in Bs]
        es = 8
    flops = float(sum(4.0 * float(m) * m * n for m, n in zip(ms, ns)))
    # algorithmic bytes: lower triangle of A read, B read, X written
    abytes = float(sum(es * (m * (m + 1) // 2) + 2 * es * m * n for m, n in zip(ms, ns)))
    return As, Bs, ms, ns, flops, abytes


def cpu_baseline_batched(As, Bs, alpha, min_seconds=3.0):
    import oracle
    reps, t0 = 0, time.perf_counter()
    while True:
        oracle.solve_batch(As, Bs, alpha)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return reps, el, oracle.num_threads()


def run_batched(args, dist, device, c64=False):
    import torch
    from paper_2608_25469_gb300 import hsma as H
    alpha = 1.5 - 0.5j
    seed = shard_seed(args.seed, dist.rank)
    As, Bs, ms, ns, flops, abytes = batched_inputs(seed, c64=c64)
    batch = len(As)
    es = 8 if c64 else 16
    code = H.C64 if c64 else H.C128
    # pack: one buffer for all A (lda = m), one for all B (ldb = m)
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)[:-1]])
    offB = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]])
    hostA = np.concatenate([a.ravel(order="F") for a in As])
    hostB = np.concatenate([b.ravel(order="F") for b in Bs])
    pinA = torch.from_numpy(hostA).pin_memory()
    pinB = torch.from_numpy(hostB).pin_memory()
    outB = torch.empty_like(pinB).pin_memory()
    dA = pinA.to(device)
    dB = pinB.to(device)
    pa = torch.from_numpy((dA.data_ptr() + offA * es).astype(np.int64)).to(device)
    pb = torch.from_numpy((dB.data_ptr() + offB * es).astype(np.int64)).to(device)
    dm = torch.from_numpy(ms.astype(np.int32)).to(device)
    dn = torch.from_numpy(ns.astype(np.int32)).to(device)
    dld = dm.clone()
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)

    def step():
        H.hsma_trsm_llnn_vbatched(code, 0, batch, dm.data_ptr(), dn.data_ptr(), alpha, pa.data_ptr(),
                                  dld.data_ptr(), pb.data_ptr(), dld.data_ptr(), 64, 64, 0, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if dist.rank == 0 else None
    if sampler:
        sampler.start()
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    torch.cuda.synchronize()
    dist.barrier()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    t1 = time.time()
    dist.barrier()
    H.hsma_trace_enable(False)
    ms_total = e0.elapsed_time(e1)
    solve_ms, solve_cnt = H.hsma_trace_read("vbatched_solve")
    phases = {ph: H.hsma_trace_read(ph) for ph in ("vbatched_schedule", "vbatched_prep", "vbatched_solve")}
    launches = H.hsma_trace_launches()
    clocks = None
    if sampler:
        sampler.mark(t0, t1)
        clocks = sampler.stop()
    ms_max = dist.max(ms_total, device=device)

    # end to end through the C ABI with host buffers: the host-buffer batch entry point
    # copies A and B in and X out, chunk by chunk, overlapped with the solves
    hm, hn = ms.astype(np.int32), ns.astype(np.int32)
    hoA, hoB = offA.astype(np.int64), offB.astype(np.int64)

    def e2e_step():
        H.hsma_trsm_llnn_vbatched_host(code, 0, batch, hm, hn, alpha, pinA.data_ptr(), hoA, pinB.data_ptr(), hoB,
                                       outB.data_ptr(), chunks=args.e2e_chunks, stream=sp)

    e2e_steps = max(1, min(args.steps, 50))
    for _ in range(2):
        e2e_step()
    torch.cuda.synchronize()
    dist.barrier()
    e0.record(st)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = dist.max(e0.elapsed_time(e1), device=device)
    total_flops = dist.sum(flops, device=device)
    value = total_flops * args.steps / (ms_max * 1e-3) / 1e9
    e2e_value = total_flops * e2e_steps / (e2e_ms * 1e-3) / 1e9

    kernel_ms = solve_ms / max(solve_cnt, 1)
    achieved = flops / (kernel_ms * 1e-3) / 1e9
    name = "c64" if c64 else "c128"
    traffic = profile_traffic(f"vbatched_solve_{name}_8192.txt", SMALL_SOURCES)
    if c64:
        # FP32 work is cheap here: the algorithmic bytes bind (HBM roofline, measured copy bandwidth)
        peaks, src = load_peaks()
        gbs = abytes / (kernel_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(gbs, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel": "vbatched_solve_kernel<cplxf>",
                "kernel_ms": round(kernel_ms, 5), "kernel_gflops": round(achieved, 2),
                "peak_source": f"HBM copy bandwidth, {src}"}
    else:
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(FP64_PEAK_GFLOPS, 1),
                "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4), "traffic": traffic,
                "kernel": "vbatched_solve_kernel<cplx>", "kernel_ms": round(kernel_ms, 5),
                "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)",
                "hbm_frac": round(abytes / (kernel_ms * 1e-3) / 1e9 / load_peaks()[0]["hbm_gbs"], 4)}
    out = {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": name, "data": "synthetic",
        "config": {"workload": f"batched_small_{name}: 8192 {'complex64' if c64 else 'complex128'} solves per "
                               "GPU, m,n ~ U{8..64}, alpha=(1.5,-0.5), non-unit, one varlen batched call per step",
                   "batch_per_gpu": batch, "seed": args.seed, "global_batch": batch * dist.world,
                   "l2": f"inputs larger than L2 ({abytes / 1e6:.0f} MB algorithmic per step)",
                   "parallelism": f"replicas x{dist.world}" if dist.world > 1 else "single GPU"},
        "roofline": roof,
        "e2e": {"value": round(e2e_value, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(hostA.nbytes + hostB.nbytes), "d2h_bytes_per_step": int(hostB.nbytes)},
        "phases_ms_per_step": {k: round(v[0] / args.steps, 5) for k, v in phases.items() if v[1]},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        wide = (lambda L: [np.asfortranarray(x.astype(np.complex128)) for x in L]) if c64 else (lambda L: L)
        reps, el, cores = cpu_baseline_batched(wide(As), wide(Bs), alpha, args.cpu_seconds)
        out["cpu_baseline"] = {"value": round(flops * reps / el / 1e9, 4), "unit": "GFLOP/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"the full 8192-instance batch, {reps} pass(es) in {el:.2f} s"}
    return out


def run_batched_lu(args, dist, device):
    """LU-factor solve as a second batched workload (the paper's motivation): 8192 complex128
    instances, m,n ~ U{8..64}; packed factors P = tril(L, -1) + triu(U); each step solves
    X = U^{-1} L^{-1} (alpha B) with the fused LU-solve batch (one launch: unit lower, then
    upper); the same work as two varlen triangular-solve launches is timed beside it."""
    import torch
    from paper_2608_25469_gb300 import hsma as H
    from paper_2608_25469_gb300 import inputs as I
    alpha = 1.5 - 0.5j
    seed = shard_seed(args.seed, dist.rank)
    ms, ns = I.batched_sizes(seed, 8192)
    Ps = []
    for b, m in enumerate(ms):
        Lf = I.gen_A(seed, int(m), I.C128, inst=b)
        Uf = I.gen_A(seed + 1, int(m), I.C128, inst=b).T
        Ps.append(np.asfortranarray(np.tril(Lf, -1) + np.triu(Uf)))
    Bs = [I.gen_B(seed, int(m), int(n), I.C128, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    batch = len(Ps)
    flops = float(sum(2 * 4.0 * float(m) * m * n for m, n in zip(ms, ns)))
    abytes = float(sum(2 * (16 * (m * (m + 1) // 2) + 2 * 16 * m * n) for m, n in zip(ms, ns)))
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)[:-1]])
    offB = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]])
    pinA = torch.from_numpy(np.concatenate([a.ravel(order="F") for a in Ps])).pin_memory()
    pinB = torch.from_numpy(np.concatenate([b.ravel(order="F") for b in Bs])).pin_memory()
    outB = torch.empty_like(pinB).pin_memory()
    dA, dB = pinA.to(device), pinB.to(device)
    pa = torch.from_numpy((dA.data_ptr() + offA * 16).astype(np.int64)).to(device)
    pb = torch.from_numpy((dB.data_ptr() + offB * 16).astype(np.int64)).to(device)
    dm = torch.from_numpy(ms.astype(np.int32)).to(device)
    dn = torch.from_numpy(ns.astype(np.int32)).to(device)
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)

    def step():
        H.hsma_getrs_vbatched(H.C128, batch, dm.data_ptr(), dn.data_ptr(), alpha, pa.data_ptr(), dm.data_ptr(), 0,
                              pb.data_ptr(), dm.data_ptr(), 64, 64, 0, sp)

    def step_two_launches():
        H.hsma_trsm_vbatched(H.C128, H.LEFT, H.LOWER, H.NO_TRANS, H.UNIT, batch, dm.data_ptr(), dn.data_ptr(), alpha,
                             pa.data_ptr(), dm.data_ptr(), pb.data_ptr(), dm.data_ptr(), 64, 64, 0, sp)
        H.hsma_trsm_vbatched(H.C128, H.LEFT, H.UPPER, H.NO_TRANS, H.NON_UNIT, batch, dm.data_ptr(), dn.data_ptr(),
                             1.0, pa.data_ptr(), dm.data_ptr(), pb.data_ptr(), dm.data_ptr(), 64, 64, 0, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if dist.rank == 0 else None
    if sampler:
        sampler.start()
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    t1 = time.time()
    H.hsma_trace_enable(False)
    ms_max = dist.max(e0.elapsed_time(e1), device=device)
    solve_ms, solve_cnt = H.hsma_trace_read("vbatched_lu")
    launches = H.hsma_trace_launches()
    clocks = None
    if sampler:
        sampler.mark(t0, t1)
        clocks = sampler.stop()
    # the same solves as two varlen triangular-solve launches, for comparison
    for _ in range(2):
        step_two_launches()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(args.steps):
        step_two_launches()
    e1.record(st)
    torch.cuda.synchronize()
    two_ms = dist.max(e0.elapsed_time(e1), device=device) / args.steps

    # end to end: A and B copied in, the fused solve, X copied out, every step
    def e2e_step():
        dA.copy_(pinA, non_blocking=True)
        dB.copy_(pinB, non_blocking=True)
        step()
        outB.copy_(dB, non_blocking=True)

    e2e_steps = max(1, min(args.steps, 50))
    e2e_step()
    torch.cuda.synchronize()
    e0.record(st)
    for _ in range(e2e_steps):
        e2e_step()
    e1.record(st)
    torch.cuda.synchronize()
    e2e_ms = dist.max(e0.elapsed_time(e1), device=device)
    total = dist.sum(flops, device=device)
    kernel_ms = solve_ms / max(solve_cnt, 1)  # one fused launch per step
    achieved = flops / (kernel_ms * 1e-3) / 1e9
    return {
        "metric": METRIC, "value": round(total * args.steps / (ms_max * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "batched_lu_c128: 8192 complex128 LU-factor solves per GPU (unit lower then upper, "
                               "one fused varlen launch), m,n ~ U{8..64}, alpha=(1.5,-0.5)",
                   "l2": f"inputs larger than L2 ({abytes / 1e6:.0f} MB algorithmic per step)"},
        "two_launches": {"ms_per_step": round(two_ms, 5),
                         "value": round(total / (two_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s"},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(FP64_PEAK_GFLOPS, 1),
                     "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
                     "traffic": profile_traffic("vbatched_lu_c128_8192.txt", SMALL_SOURCES),
                     "kernel": "vbatched_lu_kernel<cplx> (unit lower, then upper through the index map)",
                     "peak_source": "derived: 2 FP64 FMA/clk/SM x 152 SMs x 2070 MHz (nominal 1.25 TFLOP/s)"},
        "e2e": {"value": round(total * e2e_steps / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(pinA.numel() * 16 + pinB.numel() * 16),
                "d2h_bytes_per_step": int(outB.numel() * 16)},
        "gpu_launches": int(launches), "clocks": clocks,
    }


# the files that hold each profiled kernel (a summary's traffic is used only while they are unchanged)
LARGE_SOURCES = ["paper_2608_25469_gb300/csrc/blocked.cu", "paper_2608_25469_gb300/csrc/tma.cuh"]
EMU_SOURCES = ["paper_2608_25469_gb300/csrc/tc_gemm.cuh", "paper_2608_25469_gb300/csrc/tma.cuh"]
# real columns per update panel of the emulated blocked solve (the library's HSMA_EMU_PANEL_COLS)
EMU_PANEL_COLS = 2048


def run_large(args, dist, device, code, m):
    """One blocked solve per step: fp64 m = n = 16384 or complex128 m = n = 8192, alpha = 1."""
    import torch
    from paper_2608_25469_gb300 import hsma as H
    n = m
    cplx_ = code == H.C128
    dt = torch.complex128 if cplx_ else torch.float64
    es = 16 if cplx_ else 8
    seed = shard_seed(args.seed, dist.rank)
    dA = torch.empty((m, m), dtype=dt, device=device)
    dB = torch.empty((n, m), dtype=dt, device=device)
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)
    H.hsma_gen_matrix(code, 0, seed, -1, m, m, dA.data_ptr(), m, sp)
    H.hsma_gen_matrix(code, 1, seed, -1, m, n, dB.data_ptr(), m, sp)
    flops = (4.0 if cplx_ else 1.0) * float(m) * m * n
    abytes = es * (m * (m + 1) / 2 + 2.0 * m * n)
    emulated = args.fp64_products == "emulated"
    opts = H.Opts()
    opts.fp64_products = 1 if emulated else 0
    opts.nb = args.nb
    info = H.Info()

    def step():
        H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, dA.data_ptr(), m, dB.data_ptr(), m, sp, opts=opts, info=info)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    dist.barrier()
    sampler = ClockSampler(torch.cuda.current_device()) if dist.rank == 0 else None
    if sampler:
        sampler.start()
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    t0 = time.time()
    e0.record(st)
    for _ in range(args.steps):
        step()
    e1.record(st)
    torch.cuda.synchronize()
    t1 = time.time()
    H.hsma_trace_enable(False)
    ms_max = dist.max(e0.elapsed_time(e1), device=device)
    phases = {ph: H.hsma_trace_read(ph) for ph in ("diag_inverse", "copy", "slices", "solve_gemm", "update_gemm")}
    phases = {k: v for k, v in phases.items() if v[1] or k != "slices"}
    launches = H.hsma_trace_launches()
    clocks = None
    if sampler:
        sampler.mark(t0, t1)
        clocks = sampler.stop()
    upd_ms, upd_cnt = phases["update_gemm"]
    tot_phase = sum(v[0] for v in phases.values())
    # the update products' algorithmic flops: the trailing part of m^2 n not done by the solve products
    nb = info.plan.nb
    upd_flops = (4.0 if cplx_ else 1.0) * float(n) * (m * m - m * nb)
    achieved = upd_flops / (upd_ms / max(args.steps, 1) * 1e-3) / 1e9
    if emulated:
        # tensor work the emulated update products issue: 55 BF16 slice-pair
        # products of (W rows) x n x Kp each (W = 2 for complex); panels of h
        # blocks: per block an update of the panel's remaining rows (K = N_B),
        # per panel one update of the rows below it (K = h N_B)
        w = 2 if cplx_ else 1
        h = max(1, EMU_PANEL_COLS // (w * nb))
        kp = lambda k: -(-(w * k) // 64) * 64  # noqa: E731
        bf16_flops = 0.0
        for R0 in range(0, m, h * nb):
            PR = min(h * nb, m - R0)
            for r0 in range(R0, R0 + PR, nb):
                sr = min(nb, m - r0)
                bf16_flops += 55 * 2.0 * w * (R0 + PR - r0 - sr) * float(n) * kp(sr)
            bf16_flops += 55 * 2.0 * w * (m - R0 - PR) * float(n) * kp(PR)
        peaks, src = load_peaks()
        bf16_peak = peaks["bf16_tflops_sustained"] * 1e3
        bf16_rate = bf16_flops / (upd_ms / max(args.steps, 1) * 1e-3) / 1e9
    total_flops = dist.sum(flops, device=device)
    value = total_flops * args.steps / (ms_max * 1e-3) / 1e9
    name = "large_c128" if cplx_ else "large_fp64"
    # the other phases' algorithmic rates: triangular solve products (sum_r s_r(s_r+1) n flops)
    # and the diagonal-block inversion (about s_r^3/3 flops per block), x4 for complex
    kf = 4.0 if cplx_ else 1.0
    blocks = [min(nb, m - r0) for r0 in range(0, m, nb)]
    solve_flops = kf * sum(sr * (sr + 1) * float(n) for sr in blocks)
    inv_flops = kf * sum(sr ** 3 / 3.0 for sr in blocks)
    phase_rates = {}
    for ph, fl in (("solve_gemm", solve_flops), ("diag_inverse", inv_flops)):
        ms_, c = phases[ph]
        if ms_ > 0:
            rate = fl * args.steps / (ms_ * 1e-3) / 1e9
            phase_rates[ph] = {"gflops": round(rate, 2), "frac_of_fp64_peak": round(rate / FP64_PEAK_GFLOPS, 4)}
    return {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ("c128" if cplx_ else "f64") + (" (emulated: bf16 slices)" if emulated else ""),
        "data": "synthetic",
        "config": {"workload": f"{name}: one blocked solve m=n={m}, alpha=1, non-unit, N_B={nb}"
                               + (", FP64 products emulated on the BF16 tensor cores" if emulated else ""),
                   "m": m, "n": n,
                   "nb": nb, "l2": f"inputs larger than L2 ({abytes / 1e9:.2f} GB)"},
        "roofline": ({"bound": "tensor", "achieved": round(bf16_rate, 1), "peak": round(bf16_peak, 1),
                      "unit": "GFLOP/s", "frac": round(bf16_rate / bf16_peak, 4),
                      "traffic": profile_traffic(f"update_emulated_{name}.txt", EMU_SOURCES,
                                                 work=bf16_flops / max(upd_cnt / max(args.steps, 1), 1)),
                      "kernel": "tc_gemm_kernel<TC_OZ> (update_gemm, tcgen05 BF16 slice pairs)",
                      "peak_source": f"bf16 tensor (sustained), {src}",
                      "fp64_equivalent_gflops": round(achieved, 1)} if emulated else
                     {"bound": "tensor", "achieved": round(achieved, 3), "peak": round(FP64_PEAK_GFLOPS, 1),
                      "unit": "GFLOP/s", "frac": round(achieved / FP64_PEAK_GFLOPS, 4),
                      "traffic": profile_traffic(f"update_gemm_{name}.txt", LARGE_SOURCES,
                                                 work=upd_flops / max(upd_cnt / max(args.steps, 1), 1)),
                      "kernel": "gemm_kernel (update_gemm, DMMA m8n8k4)",
                      "peak_source": "derived FP64 (DMMA shares the FP64 budget): 2 FMA/clk/SM x 152 x 2070 MHz"}),
        "phases_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in phases.items()},
        "phase_share": {k: round(v[0] / tot_phase, 4) for k, v in phases.items()} if tot_phase else None,
        "phase_rates": phase_rates,
        "gpu_launches": int(launches), "clocks": clocks,
    }


def run_single64(args, dist, device):
    """Latency of one fp64 solve, m = n = 64, alpha = 1.5 (p50/p99 over the steps, graph-free launches)."""
    import torch
    from paper_2608_25469_gb300 import hsma as H
    from paper_2608_25469_gb300 import inputs as I
    A, Bm = I.gen_A(args.seed, 64, I.R64), I.gen_B(args.seed, 64, 64, I.R64)
    dA, dB = H.to_device(A), H.to_device(Bm)
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)

    def step():
        H.hsma_trsm_llnn(H.R64, 0, 64, 64, 1.5, dA.data_ptr(), 64, dB.data_ptr(), 64, sp)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    lat = []
    for _ in range(args.steps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step()
        e1.record(st)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    H.hsma_trace_enable(False)
    kms, kc = H.hsma_trace_read("small_single")
    lat = np.sort(np.array(lat))
    flops = 64.0 ** 3
    return {
        "metric": METRIC, "value": round(flops / (np.median(lat) * 1e-3) / 1e9, 4), "unit": "GFLOP/s",
        "n_gpus": 1, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(float(np.median(lat)), 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "single_fp64_64: one fp64 solve m=n=64, lda=ldb=64, alpha=1.5"},
        "latency_us": {"p50": round(float(np.percentile(lat, 50)) * 1e3, 2),
                       "p99": round(float(np.percentile(lat, 99)) * 1e3, 2),
                       "kernel_avg": round(kms / max(kc, 1) * 1e3, 2)},
    }


def run_serve(args, dist, device):
    """Serving stream: Poisson arrivals at 2000/s, m log-U[16,4096], n log-U[1,512], 70% fp64,
    16 GB admission budget, inputs generated on the device per request; p50/p99 latency."""
    import torch
    from paper_2608_25469_gb300 import hsma as H
    from paper_2608_25469_gb300 import inputs as I
    count = args.requests
    seed = shard_seed(args.seed, dist.rank)
    t_arr, ms, ns, dts = I.serving_requests(seed, count)
    flops = float(sum(I.flops_trsm(m, n, d == I.C128) for m, n, d in zip(ms, ns, dts)))
    emulated = args.fp64_products == "emulated"
    s = H.hsma_server_create(16 << 30, args.streams, H.SERVER_FP64_EMULATED if emulated else 0)
    reqs = []
    for k in range(count):
        r = H.Request()
        r.dtype, r.diag, r.m, r.n = int(dts[k]), 0, int(ms[k]), int(ns[k])
        r.alpha[0], r.alpha[1] = 1.0, 0.0
        r.gen_seed, r.gen_inst = seed, k
        reqs.append(r)
    # warm-up: the first few requests' shapes, not timed
    for k in range(min(args.warmup * 4, count)):
        H.hsma_server_submit(s, reqs[k])
    H.hsma_server_drain(s, 600.0)
    base = H.hsma_server_stats(s).submitted
    H.hsma_trace_reset()  # launch counter only: per-launch events stay off while serving
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    tickets = []
    t0 = time.perf_counter()
    for k in range(count):
        target = t0 + t_arr[k]
        while True:
            d = target - time.perf_counter()
            if d <= 0:
                break
            time.sleep(d if d > 0.002 else 0)
        tickets.append(H.hsma_server_submit(s, reqs[k]))
    H.hsma_server_drain(s, 3600.0)
    t1 = time.perf_counter()
    sampler.mark(t0, t1)
    clocks = sampler.stop()
    launches = H.hsma_trace_launches()
    lat = np.array([H.hsma_server_poll(s, t)[1] for t in tickets])
    st = H.hsma_server_stats(s)
    H.hsma_server_destroy(s)
    makespan = t1 - t0
    # the same requests one at a time with the plain solve (a sample), service time only
    k_seq = min(count, args.seq_sample)
    st_ = torch.cuda.current_stream()
    sp = int(st_.cuda_stream)
    seq = []
    seq_opts, plain_opts = H.Opts(), H.Opts()
    seq_opts.fp64_products = 1 if emulated else 0
    for k in range(k_seq):
        m, n, d = int(ms[k]), int(ns[k]), int(dts[k])
        dt = torch.complex128 if d == I.C128 else torch.float64
        A = torch.empty((m, m), dtype=dt, device=device)
        B = torch.empty((n, m), dtype=dt, device=device)
        H.hsma_gen_matrix(d, 0, seed, k, m, m, A.data_ptr(), m, sp)
        H.hsma_gen_matrix(d, 1, seed, k, m, n, B.data_ptr(), m, sp)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st_)
        # the server's rule: emulated FP64 products from m = 384
        H.hsma_trsm_llnn_ex(d, 0, m, n, 1.0, A.data_ptr(), m, B.data_ptr(), m, sp,
                            opts=seq_opts if m >= 384 else plain_opts)
        e1.record(st_)
        e1.synchronize()
        seq.append(e0.elapsed_time(e1) * 1e-3)
    seq = np.array(seq)
    seq_flops = float(sum(I.flops_trsm(m, n, d == I.C128) for m, n, d in zip(ms[:k_seq], ns[:k_seq], dts[:k_seq])))
    return {
        "metric": METRIC, "value": round(count / makespan, 2), "unit": "solves/s", "n_gpus": dist.world,
        "steps": count, "warmup": base, "ms_per_step": round(makespan * 1e3 / count, 4), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f64+c128", "data": "synthetic",
        "config": {"workload": f"serve: {count} requests, Poisson 2000/s, m log-U[16,4096], n log-U[1,512], "
                               "70% fp64 / 30% c128, 16 GB budget, device-generated inputs"
                               + ("; blocked requests with FP64 products emulated on the BF16 tensor cores"
                                  if emulated else ""),
                   "streams": args.streams},
        "gflops": round(flops / makespan / 1e9, 2), "offered_gflops": round(flops / t_arr[-1] / 1e9, 2),
        "latency_ms": {"p50": round(float(np.percentile(lat, 50)) * 1e3, 3),
                       "p99": round(float(np.percentile(lat, 99)) * 1e3, 3),
                       "max": round(float(lat.max()) * 1e3, 3)},
        "one_at_a_time": {"sample": k_seq, "solves_per_s": round(k_seq / seq.sum(), 2),
                          "gflops": round(seq_flops / seq.sum() / 1e9, 2),
                          "service_ms_p50": round(float(np.percentile(seq, 50)) * 1e3, 3),
                          "service_ms_p99": round(float(np.percentile(seq, 99)) * 1e3, 3)},
        "server": {"peak_bytes": int(st.peak_bytes_in_use), "budget_bytes": int(st.budget_bytes),
                   "batched_launches": int(st.batched_launches), "blocked_launches": int(st.blocked_launches)},
        "gpu_launches": int(launches), "clocks": clocks,
    }


def run_mixed(args, dist, device, mode):
    """m = 8192, n = 4096: FP32-result (BF16 tensor-core updates) or FP64-result (IR), beside plain fp64."""
    import torch
    from paper_2608_25469_gb300 import hsma as H
    m, n = 8192, 4096
    seed = shard_seed(args.seed, dist.rank)
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)
    A64 = torch.empty((m, m), dtype=torch.float64, device=device)
    B64 = torch.empty((n, m), dtype=torch.float64, device=device)
    H.hsma_gen_matrix(H.R64, 0, seed, -1, m, m, A64.data_ptr(), m, sp)
    H.hsma_gen_matrix(H.R64, 1, seed, -1, m, n, B64.data_ptr(), m, sp)
    flops = float(m) * m * n
    if mode == "r32":
        A = A64.float()
        B0 = B64.float()
        code = H.R32_BF16
    else:
        A = A64
        B0 = B64
        code = H.R64_IR
    B = B0.clone()
    info = H.Info()

    def step():
        B.copy_(B0)
        H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, A.data_ptr(), m, B.data_ptr(), m, sp,
                            info=info if code == H.R64_IR else None)

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    for _ in range(args.steps):
        e0.record(st)
        step()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    H.hsma_trace_enable(False)
    phases = {}
    for ph in ("diag_inverse", "copy", "solve_bf16", "solve_sgemm", "convert", "update_bf16", "residual_slices",
               "residual", "refine"):
        ms_, c = H.hsma_trace_read(ph)
        if c:
            phases[ph] = round(ms_ / args.steps, 4)
    ms_med = float(np.median(times))
    rates = {}
    if mode == "r32":
        nb = H.hsma_plan(H.R32_BF16, m, n).nb
        kp = -(-3 * nb // 64) * 64
        starts = list(range(0, m, nb))
        upd = sum(2.0 * (m - r0 - min(nb, m - r0)) * n * kp for r0 in starts)
        # solve products: six BF16 slice pairs of (s_r x n x Kd), the row tiles of the
        # triangular inverse skipping K blocks past their diagonal
        kd = -(-nb // 64) * 64
        sol = 0.0
        for r0 in starts:
            sr = min(nb, m - r0)
            sol += sum(6 * 2.0 * 128 * n * min(kd, (i0 // 256 + 1) * 256) for i0 in range(0, sr, 128))
        peaks, src = load_peaks()
        for ph, fl, pk, unit in (("update_bf16", upd, peaks["bf16_tflops"] * 1e3, "bf16 tensor (measured burst)"),
                                 ("solve_bf16", sol, peaks["bf16_tflops"] * 1e3, "bf16 tensor (measured burst)")):
            if ph in phases and phases[ph] > 0:
                rate = fl / (phases[ph] * 1e-3) / 1e9
                rates[ph] = {"gflops": round(rate, 1), "peak_gflops": round(pk, 1), "frac": round(rate / pk, 4),
                             "peak_source": f"{unit}, {src}"}
    out = {
        "metric": METRIC, "value": round(flops / (ms_med * 1e-3) / 1e9, 3), "unit": "GFLOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_med, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32(bf16 updates)" if mode == "r32" else "f64 (IR)",
        "data": "synthetic",
        "config": {"workload": f"mixed_{mode}: m=8192, n=4096, alpha=1, non-unit",
                   "step_includes": "a device copy of B (268 MB or 134 MB) to restore the input"},
        "phases_ms_per_step": phases,
        "phase_rates": rates,
    }
    if mode == "ir":
        out["ir"] = {"iterations": int(info.ir_iters), "converged": int(info.converged),
                     "residual": float(info.ir_residual)}
    # the plain fp64 solve of the same data on the same GPU (its own fp64 buffer)
    Bp = B64.clone()
    torch.cuda.synchronize()
    e0.record(st)
    H.hsma_trsm_llnn(H.R64, 0, m, n, 1.0, A64.data_ptr(), m, Bp.data_ptr(), m, sp)
    e1.record(st)
    e1.synchronize()
    pms = e0.elapsed_time(e1)
    out["plain_fp64"] = {"ms": round(pms, 3), "gflops": round(flops / (pms * 1e-3) / 1e9, 3)}
    return out


def run_reference(args, dist):
    """The oracle, as it stands, on the host cores: same metric and workload."""
    import oracle
    if dist.rank != 0:
        return None
    alpha = 1.5 - 0.5j
    As, Bs, ms, ns, flops, _ = batched_inputs(args.seed)
    # each step: a bounded sample of the batch (the first instances, about 1/8)
    k = len(As) // 8
    sflops = float(sum(4.0 * float(m) * m * n for m, n in zip(ms[:k], ns[:k])))
    for _ in range(args.warmup):
        oracle.solve_batch(As[:k], Bs[:k], alpha)
    t0 = time.perf_counter()
    for _ in range(args.steps):
        oracle.solve_batch(As[:k], Bs[:k], alpha)
    el = time.perf_counter() - t0
    v = sflops * args.steps / el / 1e9
    return {
        "impl": "reference", "metric": METRIC, "value": round(v, 4), "unit": "GFLOP/s", "n_gpus": dist.world,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(el * 1e3 / args.steps, 3),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "c128", "data": "synthetic",
        "config": {"workload": "batched_small_c128: 8192 complex128 solves, m,n ~ U{8..64}, alpha=(1.5,-0.5)",
                   "sample_per_step": f"first {k} of 8192 instances", "seed": args.seed},
        "cpu_baseline": {"value": round(v, 4), "unit": "GFLOP/s", "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"first {k} of the 8192 instances per step"},
        "e2e": {"value": round(v, 4), "unit": "GFLOP/s", "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0},
    }


def main(argv=None):
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=10)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--workload", default="batched_c128",
                    choices=["batched_c128", "batched_c64", "batched_lu_c128", "large_fp64", "large_c128",
                             "single_fp64_64", "serve", "mixed_r32", "mixed_ir"],
                    help="default: 8192 complex128 varlen solves per GPU")
    ap.add_argument("--seed", type=int, default=0)
    ap.add_argument("--cpu-seconds", type=float, default=3.0)
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--requests", type=int, default=20000)
    ap.add_argument("--seq-sample", type=int, default=1000)
    ap.add_argument("--streams", type=int, default=16)
    ap.add_argument("--m", type=int, default=0, help="large_*: m = n (default 16384 fp64, 8192 c128)")
    ap.add_argument("--fp64-products", default="dmma", choices=["dmma", "emulated"],
                    help="large_*, serve: FP64 tensor products, or FP64 emulated on the BF16 tensor cores")
    ap.add_argument("--nb", type=int, default=0, help="large_*: force N_B (0 = planner)")
    ap.add_argument("--e2e-chunks", type=int, default=0, help="batched e2e: host-buffer chunks (0 = library default)")
    args = ap.parse_args(argv)
    if args.warmup < 3:
        args.warmup = 3
    dist = Dist()
    if args.impl == "reference":
        out = run_reference(args, dist)
        if out is not None:
            print(json.dumps(out), flush=True)
        return 0
    import torch
    torch.cuda.set_device(dist.local)
    device = torch.device("cuda", dist.local)
    dist.init("nccl")
    from paper_2608_25469_gb300 import build as B
    B.build()
    from paper_2608_25469_gb300 import hsma as H
    if args.workload == "batched_c128":
        out = run_batched(args, dist, device)
    elif args.workload == "batched_c64":
        out = run_batched(args, dist, device, c64=True)
    elif args.workload == "batched_lu_c128":
        out = run_batched_lu(args, dist, device)
    elif args.workload == "large_fp64":
        out = run_large(args, dist, device, H.R64, args.m or 16384)
    elif args.workload == "large_c128":
        out = run_large(args, dist, device, H.C128, args.m or 8192)
    elif args.workload == "single_fp64_64":
        out = run_single64(args, dist, device)
    elif args.workload == "serve":
        out = run_serve(args, dist, device)
    elif args.workload in ("mixed_r32", "mixed_ir"):
        out = run_mixed(args, dist, device, args.workload.split("_")[1])
    else:
        raise SystemExit(f"unknown workload {args.workload}")
    if dist.rank == 0 and out is not None:
        print(json.dumps(out), flush=True)
    dist.close()
    return 0


if __name__ == "__main__":
    sys.exit(main())
