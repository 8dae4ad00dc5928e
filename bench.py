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
# 2 FP64 FMA per clock per SM (2 FMA x 2 flop x SMs x maximum SM clock); the
# SM count and clock are the device's own (torch device properties, nvidia-smi).
FP64_FMA_PER_CLK_PER_SM = 2
FP64_PEAK_SOURCE = "derived: 2 FP64 FMA/clk/SM x the device's SM count x its maximum SM clock (nominal 1.25 TFLOP/s)"
_fp64_peak = None


def fp64_peak_gflops():
    """2 FMA x 2 flop x SM count x maximum SM clock of the current device."""
    global _fp64_peak
    if _fp64_peak is None:
        sms, mhz = 152, 2070.0
        try:
            import torch
            sms = torch.cuda.get_device_properties(torch.cuda.current_device()).multi_processor_count
            q = subprocess.run(["nvidia-smi", f"--id={torch.cuda.current_device()}", "--query-gpu=clocks.max.sm",
                                "--format=csv,noheader,nounits"], capture_output=True, text=True, timeout=20)
            mhz = float(q.stdout.strip().splitlines()[0])
        except Exception:
            pass
        _fp64_peak = 2 * FP64_FMA_PER_CLK_PER_SM * sms * mhz * 1e6 / 1e9
    return _fp64_peak
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
    """The oracle on the whole batch, repeated for min_seconds; also returns its results."""
    import oracle
    reps, t0 = 0, time.perf_counter()
    while True:
        refs = oracle.solve_batch(As, Bs, alpha)
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            break
    return reps, el, oracle.num_threads(), refs


def batch_forward_errors(out_flat, ms, ns, refs, offB):
    """Per-instance forward errors of a packed column-major batch result."""
    import oracle
    errs = []
    for b in range(len(refs)):
        X = out_flat[offB[b]:offB[b] + ms[b] * ns[b]].reshape((ms[b], ns[b]), order="F")
        errs.append(oracle.forward_error(X, refs[b]))
    return errs


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

    # end to end through the C ABI with host buffers: the host-buffer batch entry point copies A and B in and X out,
    # chunk by chunk, overlapped with the solves.  A crosses as LAPACK-packed lower triangles (the solve reads
    # nothing else); the same call with square A is timed beside it.
    hm, hn = ms.astype(np.int32), ns.astype(np.int32)
    hoA, hoB = offA.astype(np.int64), offB.astype(np.int64)
    tri = ms.astype(np.int64) * (ms + 1) // 2
    hoT = np.concatenate([[0], np.cumsum(tri)[:-1]]).astype(np.int64)
    pinT = torch.from_numpy(np.concatenate([np.concatenate([a[j:, j] for j in range(a.shape[1])])
                                            for a in As])).pin_memory()

    def e2e_step():
        H.hsma_trsm_llnn_vbatched_host_tp(code, 0, batch, hm, hn, alpha, pinT.data_ptr(), hoT, pinB.data_ptr(), hoB,
                                          outB.data_ptr(), chunks=args.e2e_chunks, stream=sp)

    def e2e_step_square():
        H.hsma_trsm_llnn_vbatched_host(code, 0, batch, hm, hn, alpha, pinA.data_ptr(), hoA, pinB.data_ptr(), hoB,
                                       outB.data_ptr(), chunks=args.e2e_chunks, stream=sp)

    e2e_steps = max(1, min(args.steps, 50))

    def e2e_time(fn):
        for _ in range(2):
            fn()
        torch.cuda.synchronize()
        dist.barrier()
        e0.record(st)
        for _ in range(e2e_steps):
            fn()
        e1.record(st)
        torch.cuda.synchronize()
        return dist.max(e0.elapsed_time(e1), device=device)

    sq_ms = e2e_time(e2e_step_square)
    e2e_ms = e2e_time(e2e_step)  # the last call leaves X of the original data in outB
    total_flops = dist.sum(flops, device=device)
    value = total_flops * args.steps / (ms_max * 1e-3) / 1e9
    e2e_value = total_flops * e2e_steps / (e2e_ms * 1e-3) / 1e9

    kernel_ms = solve_ms / max(solve_cnt, 1)
    achieved = flops / (kernel_ms * 1e-3) / 1e9
    name = "c64" if c64 else "c128"
    # complex128 runs the column-packed batch; complex64 the per-instance kernel
    traffic = (profile_traffic("vbatched_solve_c64_8192.txt", SMALL_SOURCES) if c64 else
               profile_traffic("packed_solve_c128_8192.txt", PACKED_SOURCES, work=flops))
    if c64:
        # FP32 work is cheap here: the algorithmic bytes bind (HBM roofline, measured copy bandwidth)
        peaks, src = load_peaks()
        gbs = abytes / (kernel_ms * 1e-3) / 1e9
        roof = {"bound": "hbm", "achieved": round(gbs, 2), "peak": peaks["hbm_gbs"], "unit": "GB/s",
                "frac": round(gbs / peaks["hbm_gbs"], 4), "traffic": traffic, "kernel": "vbatched_solve_kernel<cplxf>",
                "kernel_ms": round(kernel_ms, 5), "kernel_gflops": round(achieved, 2),
                "peak_source": f"HBM copy bandwidth, {src}"}
    else:
        roof = {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp64_peak_gflops(), 1),
                "unit": "GFLOP/s", "frac": round(achieved / fp64_peak_gflops(), 4), "traffic": traffic,
                "kernel": "packed_solve_kernel<cplx>", "kernel_ms": round(kernel_ms, 5),
                "peak_source": FP64_PEAK_SOURCE,
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
                "h2d_bytes_per_step": int(pinT.numel() * pinT.element_size() + hostB.nbytes),
                "d2h_bytes_per_step": int(hostB.nbytes),
                "host_layout": "A as LAPACK-packed lower triangles (hsma_trsm_llnn_vbatched_host_tp), B and X "
                               "column-major, pinned",
                "square_A": {"value": round(total_flops * e2e_steps / (sq_ms * 1e-3) / 1e9, 3),
                             "h2d_bytes_per_step": int(hostA.nbytes + hostB.nbytes)}},
        "phases_ms_per_step": {k: round(v[0] / args.steps, 5) for k, v in phases.items() if v[1]},
        "gpu_launches": int(launches),
        "clocks": clocks,
    }
    # the last end-to-end step solved the original data: every instance against the oracle
    wide = (lambda L: [np.asfortranarray(x.astype(np.complex128)) for x in L]) if c64 else (lambda L: L)
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        reps, el, cores, refs = cpu_baseline_batched(wide(As), wide(Bs), alpha, args.cpu_seconds)
        out["cpu_baseline"] = {"value": round(flops * reps / el / 1e9, 4), "unit": "GFLOP/s", "cores": cores,
                               "kind": "oracle",
                               "sample": f"the full 8192-instance batch, {reps} pass(es) in {el:.2f} s"}
    else:
        import oracle
        refs = oracle.solve_batch(wide(As), wide(Bs), alpha)
    errs = batch_forward_errors(outB.numpy(), ms, ns, refs, offB)
    out["forward_error"] = fwd_error_record(errs, 2e-5 if c64 else 1e-12,
                                            "every instance of the batch (end-to-end result), per instance")
    return out


def run_batched_lu(args, dist, device):
    """LU-factor solve as a second batched workload (the paper's motivation): 8192 instances,
    m,n ~ U{8..64}; packed factors P = tril(L, -1) + triu(U) with getrf-style row interchanges
    (seeded LAPACK pivots, ipiv[k] uniform on k+1..m); each step solves X = U^{-1} L^{-1} P^T
    (alpha B) with the LU-solve batch (complex128: the interchange pass, then two launches of
    the column-packed batch, unit lower then upper through the index map; --lu-dtype f64:
    the fused one-launch kernel); the two triangular solves as hsma_trsm_vbatched calls are
    timed beside it."""
    import torch
    from paper_2608_25469_gb300 import hsma as H
    from paper_2608_25469_gb300 import inputs as I
    cx = args.lu_dtype == "c128"
    code = H.C128 if cx else H.R64
    es = 16 if cx else 8
    alpha = (1.5 - 0.5j) if cx else 1.5
    seed = shard_seed(args.seed, dist.rank)
    ms, ns = I.batched_sizes(seed, 8192)
    Ps = []
    for b, m in enumerate(ms):
        Lf = I.gen_A(seed, int(m), I.C128 if cx else I.R64, inst=b)
        Uf = I.gen_A(seed + 1, int(m), I.C128 if cx else I.R64, inst=b).T
        Ps.append(np.asfortranarray(np.tril(Lf, -1) + np.triu(Uf)))
    Bs = [I.gen_B(seed, int(m), int(n), I.C128 if cx else I.R64, inst=b) for b, (m, n) in enumerate(zip(ms, ns))]
    prng = np.random.default_rng(seed + 7)
    pivs = [(np.arange(int(m)) + (prng.random(int(m)) * (int(m) - np.arange(int(m)))).astype(np.int64) + 1)
            .astype(np.int32) for m in ms]
    batch = len(Ps)
    k = 4.0 if cx else 1.0
    flops = float(sum(2 * k * float(m) * m * n for m, n in zip(ms, ns)))
    abytes = float(sum(2 * (es * (m * (m + 1) // 2) + 2 * es * m * n) for m, n in zip(ms, ns)))
    offA = np.concatenate([[0], np.cumsum(ms.astype(np.int64) ** 2)[:-1]])
    offB = np.concatenate([[0], np.cumsum(ms.astype(np.int64) * ns)[:-1]])
    pinA = torch.from_numpy(np.concatenate([a.ravel(order="F") for a in Ps])).pin_memory()
    pinB = torch.from_numpy(np.concatenate([b.ravel(order="F") for b in Bs])).pin_memory()
    outB = torch.empty_like(pinB).pin_memory()
    dA, dB = pinA.to(device), pinB.to(device)
    pa = torch.from_numpy((dA.data_ptr() + offA * es).astype(np.int64)).to(device)
    pb = torch.from_numpy((dB.data_ptr() + offB * es).astype(np.int64)).to(device)
    dm = torch.from_numpy(ms.astype(np.int32)).to(device)
    dn = torch.from_numpy(ns.astype(np.int32)).to(device)
    # the pivots: one pinned array, copied with A and B every end-to-end step
    offP = np.concatenate([[0], np.cumsum(ms.astype(np.int64))[:-1]])
    pinP = torch.from_numpy(np.concatenate(pivs).astype(np.int32)).pin_memory()
    dP = pinP.to(device)
    pp = torch.from_numpy((dP.data_ptr() + offP * 4).astype(np.int64)).to(device)
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)

    def step():
        H.hsma_getrs_vbatched(code, batch, dm.data_ptr(), dn.data_ptr(), alpha, pa.data_ptr(), dm.data_ptr(),
                              pp.data_ptr(), pb.data_ptr(), dm.data_ptr(), 64, 64, 0, sp)

    def step_two_launches():  # the two triangular solves alone (no interchanges)
        H.hsma_trsm_vbatched(code, H.LEFT, H.LOWER, H.NO_TRANS, H.UNIT, batch, dm.data_ptr(), dn.data_ptr(), alpha,
                             pa.data_ptr(), dm.data_ptr(), pb.data_ptr(), dm.data_ptr(), 64, 64, 0, sp)
        H.hsma_trsm_vbatched(code, H.LEFT, H.UPPER, H.NO_TRANS, H.NON_UNIT, batch, dm.data_ptr(), dn.data_ptr(),
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
    # complex128: two packed solve launches per step; the other dtypes: one fused launch
    solve_ms, solve_cnt = H.hsma_trace_read("vbatched_solve" if cx else "vbatched_lu")
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

    # end to end: A, B and the pivots copied in, the solve, X copied out, every step
    def e2e_step():
        dA.copy_(pinA, non_blocking=True)
        dB.copy_(pinB, non_blocking=True)
        dP.copy_(pinP, non_blocking=True)
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
    kernel_ms = solve_ms / max(solve_cnt, 1)
    per_launch = flops / 2 if cx else flops  # complex128: two solve launches a step, half the flops each
    achieved = per_launch / (kernel_ms * 1e-3) / 1e9
    # the last end-to-end step solved the original data: every instance against the oracle's getrs
    # with the same pivots, which is also the timed CPU baseline
    import oracle
    t_or = time.perf_counter()
    refs = [oracle.getrs(P, piv, B, alpha) for P, piv, B in zip(Ps, pivs, Bs)]
    el_or = time.perf_counter() - t_or
    errs = batch_forward_errors(outB.numpy(), ms, ns, refs, offB)
    extra = {"forward_error": fwd_error_record(errs, 1e-12, "every instance of the batch (end-to-end result), "
                                                            "per instance, against the oracle's getrs")}
    if dist.rank == 0 and dist.world == 1 and not args.no_cpu_baseline:
        extra["cpu_baseline"] = {"value": round(flops / el_or / 1e9, 4), "unit": "GFLOP/s",
                                 "cores": oracle.num_threads(), "kind": "oracle",
                                 "sample": f"the full 8192-instance batch once, one getrs call per instance "
                                           f"({el_or:.2f} s)"}
    return {
        "metric": METRIC, "value": round(total * args.steps / (ms_max * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
        "n_gpus": dist.world, "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": args.lu_dtype, "data": "synthetic",
        "config": {"workload": (f"batched_lu_{args.lu_dtype}: 8192 "
                                f"{'complex128' if cx else 'fp64'} LU-factor solves per GPU with row "
                                "interchanges (ipiv[k] ~ U{k+1..m}; "
                                + ("the interchange pass, then unit lower and upper as two launches of the "
                                   "column-packed batch" if cx else "one fused launch: interchanges, unit lower, "
                                   "upper") + f"), m,n ~ U{{8..64}}, alpha={alpha}"),
                   "l2": f"inputs larger than L2 ({abytes / 1e6:.0f} MB algorithmic per step)"},
        "two_launches": {"ms_per_step": round(two_ms, 5),
                         "value": round(total / (two_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                         "what": "the two triangular solves as hsma_trsm_vbatched calls, no interchanges"},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp64_peak_gflops(), 1),
                     "unit": "GFLOP/s", "frac": round(achieved / fp64_peak_gflops(), 4),
                     "traffic": (profile_traffic("packed_solve_lu_upper_c128_8192.txt", PACKED_SOURCES,
                                                 work=flops / 2) if cx else
                                 profile_traffic("vbatched_lu_f64_8192.txt", SMALL_SOURCES)),
                     "kernel": ("packed_solve_kernel<cplx> (two launches a step: unit lower, then upper "
                                "through the index map; achieved over both)" if cx else
                                "vbatched_lu_kernel<double> (interchanges, unit lower and upper in one launch)"),
                     "kernel_ms": round(kernel_ms, 5),
                     "peak_source": FP64_PEAK_SOURCE},
        "e2e": {"value": round(total * e2e_steps / (e2e_ms * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(pinA.numel() * es + pinB.numel() * es + pinP.numel() * 4),
                "d2h_bytes_per_step": int(outB.numel() * es)},
        "gpu_launches": int(launches), "clocks": clocks,
        **extra,
    }


# the files that hold each profiled kernel (a summary's traffic is used only while they are unchanged)
LARGE_SOURCES = ["paper_2608_25469_gb300/csrc/blocked.cu", "paper_2608_25469_gb300/csrc/tma.cuh"]
EMU_SOURCES = ["paper_2608_25469_gb300/csrc/tc_gemm.cuh", "paper_2608_25469_gb300/csrc/tma.cuh"]
# real columns per update panel of the emulated blocked solve when the plan reports none
EMU_PANEL_COLS = 2048


def sample_cols(n, k):
    """k evenly spaced column indices of an n-column B (all of them when n <= k)."""
    return np.unique(np.linspace(0, n - 1, min(n, k)).round().astype(np.int64))


def dense_checks(dA, dB, regen_B, solve, alpha, cplx_, cols, tol, a64=None, b64_cols=None, cpu_cols=8):
    """For one dense solve on the device (dA: (m, m) tensor holding column-major A, dB:
    (n, m) tensor holding column-major B): regenerate B, solve once, and compare the
    sampled columns with the FP64 oracle (exact per column); then time the oracle on
    `cpu_cols` of those columns.  a64 / b64_cols: the FP64 data the oracle solves when
    the device works on rounded copies (FP32-result mode)."""
    import torch
    import oracle
    regen_B()
    torch.cuda.synchronize()
    if b64_cols is None:
        b64_cols = np.asfortranarray(dB[torch.as_tensor(cols, device=dB.device)].cpu().numpy().T)
        b64_cols = b64_cols.astype(np.complex128 if cplx_ else np.float64)
    solve()
    torch.cuda.synchronize()
    X = dB[torch.as_tensor(cols, device=dB.device)].cpu().numpy().T
    X = np.asfortranarray(X.astype(np.complex128 if cplx_ else np.float64))
    if a64 is None:
        a64 = np.asfortranarray(dA.cpu().numpy().T)
    ref = oracle.solve_cols(a64, b64_cols, alpha, np.arange(b64_cols.shape[1]))
    errs = [oracle.forward_error(X[:, k:k + 1], ref[:, k:k + 1]) for k in range(len(cols))]
    whole = oracle.forward_error(X, ref)
    sub = np.asfortranarray(b64_cols[:, :cpu_cols])
    t0 = time.perf_counter()
    oracle.solve_cols(a64, sub, alpha, np.arange(sub.shape[1]))
    cel = time.perf_counter() - t0
    m = a64.shape[1]
    kf = 4.0 if cplx_ else 1.0
    rec = fwd_error_record(errs, tol, f"{len(cols)} evenly spaced columns of a fresh solve (per column); "
                                     f"over the whole sample {whole:.3e}")
    cpu = {"value": round(kf * m * m * sub.shape[1] / cel / 1e9, 4), "unit": "GFLOP/s", "cores": oracle.num_threads(),
           "kind": "oracle", "sample": f"{sub.shape[1]} columns of the full-size problem in {cel:.2f} s"}
    return rec, cpu, a64


def e2e_dense(dA, dB, solve, flops, reps=1, extra=None):
    """End to end with host buffers: A and B copied from pinned host memory, the solve, X
    copied back, every step; returns the e2e record."""
    import torch
    st = torch.cuda.current_stream()
    hA = torch.empty(dA.shape, dtype=dA.dtype, pin_memory=True)
    hA.copy_(dA)
    hB = torch.empty(dB.shape, dtype=dB.dtype, pin_memory=True)
    hB.copy_(dB)
    hX = torch.empty_like(hB, pin_memory=True)
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(reps):
        dA.copy_(hA, non_blocking=True)
        dB.copy_(hB, non_blocking=True)
        solve()
        hX.copy_(dB, non_blocking=True)
    e1.record(st)
    torch.cuda.synchronize()
    ms_ = e0.elapsed_time(e1) / reps
    rec = {"value": round(flops / (ms_ * 1e-3) / 1e9, 3), "unit": "GFLOP/s",
           "h2d_bytes_per_step": int(hA.numel() * hA.element_size() + hB.numel() * hB.element_size()),
           "d2h_bytes_per_step": int(hX.numel() * hX.element_size()), "ms_per_step": round(ms_, 3)}
    if extra:
        rec.update(extra)
    return rec


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
        h = max(1, (info.plan.panel_cols or EMU_PANEL_COLS) // (w * nb))
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
            phase_rates[ph] = {"gflops": round(rate, 2), "frac_of_fp64_peak": round(rate / fp64_peak_gflops(), 4)}
    # a fresh solve checked on 64 sampled columns; the oracle timed on 8 of them;
    # then one step end to end from pinned host buffers
    regen = lambda: H.hsma_gen_matrix(code, 1, seed, -1, m, n, dB.data_ptr(), m, sp)  # noqa: E731
    ferr, cpu, _ = dense_checks(dA, dB, regen, step, 1.0, cplx_, sample_cols(n, 64), 1e-12)
    regen()
    e2e = e2e_dense(dA, dB, step, flops)
    return {
        "metric": METRIC, "value": round(value, 3), "unit": "GFLOP/s", "n_gpus": dist.world, "steps": args.steps,
        "warmup": args.warmup, "ms_per_step": round(ms_max / args.steps, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": ("c128" if cplx_ else "f64") + (" (emulated: bf16 slices)" if emulated else ""),
        "data": "synthetic",
        "config": {"workload": f"{name}: one blocked solve m=n={m}, alpha=1, non-unit, N_B={nb}"
                               + (", FP64 products emulated on the BF16 tensor cores" if emulated else ""),
                   "m": m, "n": n, "nb": nb,
                   "plan": {"tile": info.plan.tile, "split_k": info.plan.split_k, "looking": info.plan.looking,
                            "panel_cols": info.plan.panel_cols},
                   "l2": f"inputs larger than L2 ({abytes / 1e9:.2f} GB)"},
        "roofline": ({"bound": "tensor", "achieved": round(bf16_rate, 1), "peak": round(bf16_peak, 1),
                      "unit": "GFLOP/s", "frac": round(bf16_rate / bf16_peak, 4),
                      "traffic": profile_traffic(f"update_emulated_{name}.txt", EMU_SOURCES,
                                                 work=bf16_flops / max(upd_cnt / max(args.steps, 1), 1)),
                      "kernel": "tc_gemm_kernel<TC_OZ> (update_gemm, tcgen05 BF16 slice pairs)",
                      "peak_source": f"bf16 tensor (sustained), {src}",
                      "fp64_equivalent_gflops": round(achieved, 1)} if emulated else
                     {"bound": "tensor", "achieved": round(achieved, 3), "peak": round(fp64_peak_gflops(), 1),
                      "unit": "GFLOP/s", "frac": round(achieved / fp64_peak_gflops(), 4),
                      "traffic": profile_traffic(f"update_gemm_{name}.txt", LARGE_SOURCES,
                                                 work=upd_flops / max(upd_cnt / max(args.steps, 1), 1)),
                      "kernel": "gemm_kernel (update_gemm, DMMA m8n8k4)",
                      "peak_source": FP64_PEAK_SOURCE + "; DMMA shares the FP64 budget"}),
        "phases_ms_per_step": {k: round(v[0] / args.steps, 3) for k, v in phases.items()},
        "phase_share": {k: round(v[0] / tot_phase, 4) for k, v in phases.items()} if tot_phase else None,
        "phase_rates": phase_rates,
        "forward_error": ferr, "cpu_baseline": cpu, "e2e": e2e,
        "gpu_launches": int(launches), "clocks": clocks,
    }


def fwd_error_record(errs, tol, sample):
    """Measured relative Frobenius forward errors against the FP64 oracle."""
    errs = np.asarray(errs, dtype=np.float64)
    return {"max": float(errs.max()), "median": float(np.median(errs)), "tolerance": tol,
            "within": bool(errs.max() <= tol), "vs": "FP64 oracle (oracle/trsm_oracle.c)", "sample": sample}


def timed_oracle(fn, min_seconds):
    """Run fn until min_seconds have passed; returns (repetitions, seconds)."""
    reps, t0 = 0, time.perf_counter()
    while True:
        fn()
        reps += 1
        el = time.perf_counter() - t0
        if el >= min_seconds:
            return reps, el


def run_single64(args, dist, device):
    """One fp64 solve, m = n = 64, lda = ldb = 64, alpha = 1.5, seed 0.  value: GFLOP/s at the
    p50 latency of CUDA-graph replays of the solve; also the per-launch latency, the same
    problem replicated 8192 times in one batched call, and the host-buffer round trip."""
    import torch
    import oracle
    from paper_2608_25469_gb300 import hsma as H
    from paper_2608_25469_gb300 import inputs as I
    m = n = 64
    alpha = 1.5
    A, Bm = I.gen_A(args.seed, m, I.R64), I.gen_B(args.seed, m, n, I.R64)
    flops = float(m) * m * n
    dA, dB = H.to_device(A), H.to_device(Bm)
    dB0 = dB.clone()
    st = torch.cuda.current_stream()
    sp = int(st.cuda_stream)

    def step(stream_ptr):
        H.hsma_trsm_llnn(H.R64, 0, m, n, alpha, dA.data_ptr(), m, dB.data_ptr(), m, stream_ptr)

    for _ in range(args.warmup):
        step(sp)
    torch.cuda.synchronize()
    # the result of one solve of the original data, against the oracle
    dB.copy_(dB0)
    step(sp)
    torch.cuda.synchronize()
    ref = oracle.solve(A, Bm, alpha)
    ferr = oracle.forward_error(H.from_device(dB), ref)
    # per-launch latency (events around each call)
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    reps = max(args.steps, 200)
    lat = []
    for k in range(reps):
        if k % 100 == 0:
            dB.copy_(dB0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        step(sp)
        e1.record(st)
        e1.synchronize()
        lat.append(e0.elapsed_time(e1))
    H.hsma_trace_enable(False)
    kms, kc = H.hsma_trace_read("small_single")
    kernel_us = kms / max(kc, 1) * 1e3
    # CUDA-graph replays of the same call
    g = torch.cuda.CUDAGraph()
    cs = torch.cuda.Stream()
    cs.wait_stream(st)
    with torch.cuda.stream(cs):
        step(int(cs.cuda_stream))
    torch.cuda.synchronize()
    cap0 = H.hsma_trace_launches()
    with torch.cuda.graph(g):
        step(int(torch.cuda.current_stream().cuda_stream))
    torch.cuda.synchronize()
    per_graph = H.hsma_trace_launches() - cap0  # the library's kernels recorded in the graph
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    glat = []
    t0 = time.time()
    for k in range(reps * 5):
        if k % 100 == 0:
            dB.copy_(dB0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        g.replay()
        e1.record(st)
        e1.synchronize()
        glat.append(e0.elapsed_time(e1))
    t1 = time.time()
    sampler.mark(t0, t1)
    clocks = sampler.stop()
    launches = per_graph * len(glat)  # graph replays do not pass the host launch sites
    lat, glat = np.sort(np.array(lat)), np.sort(np.array(glat))
    p50 = float(np.percentile(glat, 50))
    # the same problem replicated 8192 times in one batched call (B copies; A shared)
    R = 8192
    bigB = dB0.repeat(R, 1).contiguous()  # R copies of the 64 x 64 block, column-major each
    pa = torch.full((R,), dA.data_ptr(), dtype=torch.int64, device=device)
    pb = (bigB.data_ptr() + torch.arange(R, dtype=torch.int64, device=device) * (m * n * 8)).contiguous()
    dm = torch.full((R,), m, dtype=torch.int32, device=device)

    def rep_step():
        H.hsma_trsm_llnn_vbatched(H.R64, 0, R, dm.data_ptr(), dm.data_ptr(), alpha, pa.data_ptr(), dm.data_ptr(),
                                  pb.data_ptr(), dm.data_ptr(), 64, 64, 0, sp)

    for _ in range(3):
        rep_step()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    e0.record(st)
    for _ in range(10):
        rep_step()
    e1.record(st)
    torch.cuda.synchronize()
    rep_ms = e0.elapsed_time(e1) / 10
    # end to end: A and B from pinned host memory, the solve, X back, every call
    hA = torch.from_numpy(np.asfortranarray(A).ravel(order="F")).pin_memory()
    hB = torch.from_numpy(np.asfortranarray(Bm).ravel(order="F")).pin_memory()
    hX = torch.empty_like(hB).pin_memory()
    fA, fB = dA.view(-1), dB.view(-1)

    def e2e_step():
        fA.copy_(hA, non_blocking=True)
        fB.copy_(hB, non_blocking=True)
        step(sp)
        hX.copy_(fB, non_blocking=True)

    for _ in range(3):
        e2e_step()
    torch.cuda.synchronize()
    elat = []
    for _ in range(reps):
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record(st)
        e2e_step()
        e1.record(st)
        e1.synchronize()
        elat.append(e0.elapsed_time(e1))
    e2e_p50 = float(np.percentile(elat, 50))
    # the oracle on the host cores, the same solve repeated
    creps, cel = timed_oracle(lambda: oracle.solve(A, Bm, alpha), min(args.cpu_seconds, 2.0))
    # dependent chain of the substitution: one FP64 FMA latency (64 cycles) and one
    # shuffle (about 30 cycles) per row, at the sampled SM clock
    mhz = (clocks or {}).get("sm_mhz") or 2070.0
    chain_us = (m - 1) * (64 + 30) / mhz
    achieved = flops / (kernel_us * 1e-6) / 1e9
    return {
        "metric": METRIC, "value": round(flops / (p50 * 1e-3) / 1e9, 4), "unit": "GFLOP/s",
        "n_gpus": 1, "steps": reps * 5, "warmup": args.warmup, "ms_per_step": round(p50, 5),
        "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
        "config": {"workload": "single_fp64_64: one fp64 solve m=n=64, lda=ldb=64, alpha=1.5, seed 0; value at "
                               "the p50 latency of CUDA-graph replays",
                   "l2": "82 KB working set (latency-bound: L2 state does not matter)"},
        "latency_us": {"graph_p50": round(p50 * 1e3, 2), "graph_p99": round(float(np.percentile(glat, 99)) * 1e3, 2),
                       "launch_p50": round(float(np.percentile(lat, 50)) * 1e3, 2),
                       "launch_p99": round(float(np.percentile(lat, 99)) * 1e3, 2),
                       "kernel_avg": round(kernel_us, 2), "dependent_chain_estimate": round(chain_us, 2)},
        "replicated_8192": {"ms": round(rep_ms, 4), "gflops": round(R * flops / (rep_ms * 1e-3) / 1e9, 2),
                            "how": "the same 64 x 64 problem 8192 times in one varlen batched call"},
        "roofline": {"bound": "alu", "achieved": round(achieved, 3), "peak": round(fp64_peak_gflops(), 1),
                     "unit": "GFLOP/s", "frac": round(achieved / fp64_peak_gflops(), 5),
                     "traffic": profile_traffic("small_single_fp64_64.txt", SMALL_SOURCES),
                     "kernel": "small_single_kernel<double>",
                     "peak_source": FP64_PEAK_SOURCE,
                     "note": "one 64 x 64 solve cannot fill the GPU: its bound is the 63-step dependent chain "
                             "(dependent_chain_estimate), not the FP64 throughput"},
        "e2e": {"value": round(flops / (e2e_p50 * 1e-3) / 1e9, 4), "unit": "GFLOP/s",
                "h2d_bytes_per_step": int(hA.numel() * 8 + hB.numel() * 8), "d2h_bytes_per_step": int(hX.numel() * 8),
                "latency_us_p50": round(e2e_p50 * 1e3, 2)},
        "cpu_baseline": {"value": round(flops * creps / cel / 1e9, 4), "unit": "GFLOP/s",
                         "cores": oracle.num_threads(), "kind": "oracle",
                         "sample": f"the same solve, {creps} times in {cel:.2f} s"},
        "forward_error": fwd_error_record([ferr], 1e-12, "the full 64 x 64 result"),
        "gpu_launches": int(launches), "clocks": clocks,
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
    # a seeded 1% sample of the requests returns its X to host memory for the oracle check
    sample = np.arange(seed % 100, count, 100)
    xbuf = {}
    for k in sample:
        dt = torch.complex128 if int(dts[k]) == I.C128 else torch.float64
        xbuf[int(k)] = torch.empty((int(ns[k]), int(ms[k])), dtype=dt, pin_memory=True)
        reqs[k].X_host, reqs[k].ldx = xbuf[int(k)].data_ptr(), int(ms[k])
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
    # the sample against the oracle (inputs regenerated by the same device generator)
    import oracle
    errs, ot, ofl = [], 0.0, 0.0
    for k in sample:
        m, n, d = int(ms[k]), int(ns[k]), int(dts[k])
        dt = torch.complex128 if d == I.C128 else torch.float64
        A = torch.empty((m, m), dtype=dt, device=device)
        B = torch.empty((n, m), dtype=dt, device=device)
        H.hsma_gen_matrix(d, 0, seed, int(k), m, m, A.data_ptr(), m, sp)
        H.hsma_gen_matrix(d, 1, seed, int(k), m, n, B.data_ptr(), m, sp)
        torch.cuda.synchronize()
        Ah, Bh = np.asfortranarray(A.cpu().numpy().T), np.asfortranarray(B.cpu().numpy().T)
        t_ = time.perf_counter()
        ref = oracle.solve(Ah, Bh, 1.0)
        ot += time.perf_counter() - t_
        ofl += I.flops_trsm(m, n, d == I.C128)
        errs.append(oracle.forward_error(np.asfortranarray(xbuf[int(k)].numpy().T), ref))
    ferr = fwd_error_record(errs, 1e-12, f"seeded 1% of the requests ({len(sample)}), X returned to host memory "
                                         "by the server, per request")
    cpu = {"value": round(len(sample) / ot, 3), "unit": "solves/s", "gflops": round(ofl / ot / 1e9, 3),
           "cores": oracle.num_threads(), "kind": "oracle",
           "sample": f"the same {len(sample)} sampled requests, solved in {ot:.2f} s"}
    e2e = serve_e2e(args, H, I, seed, t_arr, ms, ns, dts, emulated, device)
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
        "forward_error": ferr, "cpu_baseline": cpu, "e2e": e2e,
        "roofline": {"bound": "alu", "achieved": round(flops / makespan / 1e9, 2),
                     "peak": round(fp64_peak_gflops(), 1), "unit": "GFLOP/s",
                     "frac": round(flops / makespan / 1e9 / fp64_peak_gflops(), 4), "traffic": None,
                     "kernel": "whole stream (arrival-paced: the offered load, not the GPU, sets the rate)",
                     "peak_source": FP64_PEAK_SOURCE},
        "gpu_launches": int(launches), "clocks": clocks,
    }


def serve_e2e(args, H, I, seed, t_arr, ms, ns, dts, emulated, device, count=2000):
    """The first `count` requests of the stream, paced the same way, with every request's A
    and B copied by the server from pinned host memory and X copied back to pinned host
    memory.  The sources are shared: one generated 4096 x 4096 triangle and 4096 x 512 B per
    dtype, each request reading its leading m x m / m x n block (lda = 4096)."""
    import torch
    count = min(count, len(ms))
    src = {}
    for d in (I.R64, I.C128):
        dt = torch.complex128 if d == I.C128 else torch.float64
        A = torch.empty((4096, 4096), dtype=dt, device=device)
        B = torch.empty((512, 4096), dtype=dt, device=device)
        H.hsma_gen_matrix(d, 0, seed + 7, -1, 4096, 4096, A.data_ptr(), 4096, 0)
        H.hsma_gen_matrix(d, 1, seed + 7, -1, 4096, 512, B.data_ptr(), 4096, 0)
        torch.cuda.synchronize()
        hA = torch.empty_like(A, device="cpu", pin_memory=True)
        hB = torch.empty_like(B, device="cpu", pin_memory=True)
        hA.copy_(A)
        hB.copy_(B)
        src[d] = (hA, hB)
    es = [16 if int(d) == I.C128 else 8 for d in dts[:count]]
    xsz = [int(ms[k]) * int(ns[k]) * es[k] for k in range(count)]
    arena = torch.empty(sum(xsz), dtype=torch.uint8, pin_memory=True)
    off = np.concatenate([[0], np.cumsum(xsz)[:-1]])
    s = H.hsma_server_create(16 << 30, args.streams, H.SERVER_FP64_EMULATED if emulated else 0)
    reqs = []
    for k in range(count):
        r = H.Request()
        d = int(dts[k])
        r.dtype, r.diag, r.m, r.n = d, 0, int(ms[k]), int(ns[k])
        r.alpha[0], r.alpha[1] = 1.0, 0.0
        r.A_host, r.lda = src[d][0].data_ptr(), 4096
        r.B_host, r.ldb = src[d][1].data_ptr(), 4096
        r.X_host, r.ldx = arena.data_ptr() + int(off[k]), int(ms[k])
        reqs.append(r)
    for k in range(min(8, count)):  # warm-up
        H.hsma_server_submit(s, reqs[k])
    H.hsma_server_drain(s, 600.0)
    tickets = []
    t0 = time.perf_counter()
    for k in range(count):
        target = t0 + (t_arr[k] - t_arr[0])
        while True:
            dl = target - time.perf_counter()
            if dl <= 0:
                break
            time.sleep(dl if dl > 0.002 else 0)
        tickets.append(H.hsma_server_submit(s, reqs[k]))
    H.hsma_server_drain(s, 3600.0)
    t1 = time.perf_counter()
    lat = np.array([H.hsma_server_poll(s, t)[1] for t in tickets])
    H.hsma_server_destroy(s)
    h2d = sum(int(ms[k]) * (int(ms[k]) + int(ns[k])) * es[k] for k in range(count))
    return {"value": round(count / (t1 - t0), 2), "unit": "solves/s", "requests": count,
            "h2d_bytes_per_step": int(h2d / count), "d2h_bytes_per_step": int(sum(xsz) / count),
            "per": "request (a step of this workload is one request)",
            "latency_ms": {"p50": round(float(np.percentile(lat, 50)) * 1e3, 3),
                           "p99": round(float(np.percentile(lat, 99)) * 1e3, 3)},
            "sources": "pinned host buffers (shared read-only inputs per dtype, one output region per request)"}


def ir_residual_bf16_flops(m, n, chunk=1024, tile=128, pairs=55):
    """BF16 slice-pair flops of one emulated refinement residual R = alpha B - L X: K chunks
    of `chunk` columns of L; a chunk starting at c0 multiplies rows c0.. of L, row tile t
    (of `tile` rows) needing K up to its own last row (64-padded)."""
    tot = 0.0
    for c0 in range(0, m, chunk):
        kc = min(chunk, m - c0)
        K = -(-kc // 64) * 64
        M = m - c0
        for pm in range(-(-M // tile)):
            rows = min(tile, M - pm * tile)
            kall = -(-min(K, (pm + 1) * tile) // 64) * 64
            tot += pairs * 2.0 * rows * n * kall
    return tot


def run_mixed(args, dist, device, mode):
    """m = 8192, n = 4096, alpha = 1: the FP32-result mode (split-BF16 tensor-core updates)
    or the FP64-result mode (FP32-result solves + FP64 refinement), beside the plain FP64
    solve on the same GPU with FP64 tensor products (DMMA) and with FP64 products emulated
    on the BF16 tensor cores."""
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
        A, B0, code, tol = A64.float(), B64.float(), H.R32_BF16, 2e-5
    else:
        A, B0, code, tol = A64, B64, H.R64_IR, 1e-12
    B = B0.clone()
    info = H.Info()

    def solve():
        H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, A.data_ptr(), m, B.data_ptr(), m, sp,
                            info=info if code == H.R64_IR else None)

    def step():
        B.copy_(B0)
        solve()

    for _ in range(args.warmup):
        step()
    torch.cuda.synchronize()
    sampler = ClockSampler(torch.cuda.current_device())
    sampler.start()
    H.hsma_trace_reset()
    H.hsma_trace_enable(True)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    times = []
    t0 = time.time()
    for _ in range(args.steps):
        e0.record(st)
        step()
        e1.record(st)
        e1.synchronize()
        times.append(e0.elapsed_time(e1))
    t1 = time.time()
    H.hsma_trace_enable(False)
    sampler.mark(t0, t1)
    clocks = sampler.stop()
    launches = H.hsma_trace_launches()
    phases, counts = {}, {}
    for ph in ("diag_inverse", "copy", "solve_bf16", "solve_sgemm", "convert", "update_bf16", "residual_slices",
               "residual", "refine"):
        ms_, c = H.hsma_trace_read(ph)
        if c:
            phases[ph] = round(ms_ / args.steps, 4)
            counts[ph] = c / args.steps
    ms_med = float(np.median(times))
    peaks, src = load_peaks()
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
        for ph, fl in (("update_bf16", upd), ("solve_bf16", sol)):
            if ph in phases and phases[ph] > 0:
                rate = fl / (phases[ph] * 1e-3) / 1e9
                rates[ph] = {"gflops": round(rate, 1), "frac_of_bf16_burst": round(rate / (peaks["bf16_tflops"] * 1e3), 4)}
        ups = counts.get("update_bf16", 1)
        kernel_ms = phases.get("update_bf16", 0.0) / max(ups, 1)
        ach = upd / max(ups, 1) / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else 0.0
        pk = peaks["bf16_tflops"] * 1e3
        roof = {"bound": "tensor", "achieved": round(ach, 1), "peak": round(pk, 1), "unit": "GFLOP/s",
                "frac": round(ach / pk, 4),
                "traffic": profile_traffic("tc_f32_update_r32_8192x4096.txt", EMU_SOURCES, work=upd / max(ups, 1)),
                "kernel": "tc_gemm_kernel<TC_F32> (update_bf16: split-BF16 trailing update, FP32 accumulate)",
                "kernel_ms": round(kernel_ms, 5), "peak_source": f"bf16 tensor (measured burst), {src}"}
    else:
        evals = int(info.ir_iters) + 1  # residual evaluations that did work (one per check)
        res_fl = ir_residual_bf16_flops(m, n)
        rcnt = counts.get("residual", 1)  # launches per step (one per K chunk and evaluation)
        kernel_ms = phases.get("residual", 0.0) / max(rcnt, 1)
        ach = res_fl * evals / max(rcnt, 1) / (kernel_ms * 1e-3) / 1e9 if kernel_ms > 0 else 0.0
        pk = peaks["bf16_tflops_sustained"] * 1e3
        roof = {"bound": "tensor", "achieved": round(ach, 1), "peak": round(pk, 1), "unit": "GFLOP/s",
                "frac": round(ach / pk, 4),
                "traffic": profile_traffic("residual_emulated_ir_8192x4096.txt", EMU_SOURCES,
                                           work=res_fl * evals / max(rcnt, 1)),
                "kernel": "tc_gemm_kernel<TC_OZ> (residual: 55 BF16 slice pairs per K chunk of 1024)",
                "kernel_ms": round(kernel_ms, 5), "residual_evaluations": evals,
                "peak_source": f"bf16 tensor (measured sustained), {src}"}
        if "residual" in phases:
            rates["residual"] = {"fp64_equivalent_gflops": round(flops * evals / (phases["residual"] * 1e-3) / 1e9, 1)}
    # the same solve checked against the oracle on sampled columns (FP64 data)
    a64 = np.asfortranarray(A64.cpu().numpy().T)
    cols = sample_cols(n, 64)
    b64c = np.asfortranarray(B64[torch.as_tensor(cols, device=device)].cpu().numpy().T)
    ferr, cpu, _ = dense_checks(A, B, lambda: B.copy_(B0), solve, 1.0, False, cols, tol, a64=a64, b64_cols=b64c)
    # comparators on the same GPU: the plain FP64 solve with DMMA products and with
    # emulated FP64 products, each timed and checked the same way
    comps = {}
    for label, fp in (("plain_fp64_dmma", 0), ("plain_fp64_emulated", 1)):
        o = H.Opts()
        o.fp64_products = fp
        Bp = B64.clone()

        def psolve(o=o, Bp=Bp):
            H.hsma_trsm_llnn_ex(H.R64, 0, m, n, 1.0, A64.data_ptr(), m, Bp.data_ptr(), m, sp, opts=o)

        reps = 1 if fp == 0 else 3
        psolve()
        torch.cuda.synchronize()
        e0.record(st)
        for _ in range(reps):
            Bp.copy_(B64)
            psolve()
        e1.record(st)
        torch.cuda.synchronize()
        pms = e0.elapsed_time(e1) / reps
        pe, _, _ = dense_checks(A64, Bp, lambda Bp=Bp: Bp.copy_(B64), psolve, 1.0, False, cols, 1e-12, a64=a64,
                                b64_cols=b64c)
        comps[label] = {"ms": round(pms, 3), "gflops": round(flops / (pms * 1e-3) / 1e9, 3),
                        "forward_error_max": pe["max"], "includes": "a device copy of B"}
    B.copy_(B0)
    e2e = e2e_dense(A, B, solve, flops, extra={"includes": "A (lower triangle read) and B in, X out, every step"})
    out = {
        "metric": METRIC, "value": round(flops / (ms_med * 1e-3) / 1e9, 3), "unit": "GFLOP/s", "n_gpus": 1,
        "steps": args.steps, "warmup": args.warmup, "ms_per_step": round(ms_med, 3), "higher_is_better": True,
        "scaling": "weak", "vs_baseline": None, "dtype": "f32 (split-bf16 updates)" if mode == "r32" else "f64 (IR)",
        "data": "synthetic",
        "config": {"workload": f"mixed_{mode}: m=8192, n=4096, alpha=1, non-unit, seed 0",
                   "step_includes": "a device copy of B (268 MB or 134 MB) to restore the input",
                   "l2": "inputs larger than L2"},
        "phases_ms_per_step": phases, "phase_rates": rates, "roofline": roof,
        "forward_error": ferr, "cpu_baseline": cpu, "e2e": e2e, "comparators": comps,
        "gpu_launches": int(launches), "clocks": clocks,
    }
    if mode == "ir":
        out["ir"] = {"iterations": int(info.ir_iters), "converged": int(info.converged),
                     "residual": float(info.ir_residual)}
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
    ap.add_argument("--lu-dtype", default="c128", choices=["c128", "f64"],
                    help="batched_lu_c128: element type of the LU-factor batch (f64 runs the fused kernel)")
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
