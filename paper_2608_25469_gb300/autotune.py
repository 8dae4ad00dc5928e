"""Offline configuration profiling for the blocked path (Section 4.3.2).

For every (dtype, m, n) point of a grid, time the blocked solve over the
configuration space and keep the fastest, then write the "scale x dtype ->
configuration" table: ``csrc/tuning_table.inc`` (compiled into the library)
plus ``tuning/tuning_gb300.txt`` (loadable at run time with
``hsma_tuning_load``) and ``tuning/tuning_gb300.json`` (every candidate's
time).  At run time the planner picks the entry nearest to the input in
(log m, log n).

Configuration space per dtype:

* R64 / C128 with FP64 tensor products (DMMA): the diagonal block size N_B,
  the product tile (64 x 64, 128 x 16, 128 x 8 rows x columns, or the rule by
  n), split K (when the tiles leave SMs idle, or never) and the update
  direction (right-looking, or the paper's left-looking form).  Searched in
  stages: N_B with the default rest, then the tile, split K and direction one
  at a time from the best so far (each stage keeps what it measured fastest).
* R64 / C128 with FP64 products emulated on the BF16 tensor cores (table keys
  dtype + 10): N_B x the update-panel width.
* R32_BF16 (FP32-result mode, also used by R64_IR and R32): N_B.

    python -m paper_2608_25469_gb300.autotune [--quick] [--out-dir DIR]

Needs a GPU.  Inputs come from the device-side seeded generator.
"""
from __future__ import annotations

import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
NBS = (32, 64, 128, 256, 512)
TILES = (1, 2, 3)          # HSMA_TILE_64x64, _128x16, _128x8 (0 = the rule by n)
EMU_NBS = (256, 512)
PANELS = (1024, 2048, 3072, 4096)
EMU = 10                   # table key offset of the emulated-products entries

GRID = {
    0: [(m, n) for m in (128, 512, 2048, 8192) for n in (16, 256, 4096)] + [(16384, 16384)],
    1: [(m, n) for m in (128, 512, 2048) for n in (16, 256, 2048)] + [(8192, 8192)],
    2: [(m, n) for m in (128, 512, 2048, 8192) for n in (16, 256, 4096)],
    EMU + 0: [(2048, 2048), (8192, 4096), (16384, 16384)],
    EMU + 1: [(2048, 2048), (4096, 4096), (8192, 8192)],
}
QUICK = {0: [(512, 256), (4096, 4096)], 1: [(512, 256), (2048, 2048)], 2: [(1024, 256), (8192, 4096)],
         EMU + 0: [(4096, 4096)], EMU + 1: [(2048, 2048)]}


class Problem:
    """Device inputs of one (dtype, m, n) point and a timed solve with given options."""

    def __init__(self, H, torch, code, m, n):
        base = code % EMU
        gen_code = 1 if base == 1 else 0
        self.H, self.torch, self.m, self.n = H, torch, m, n
        self.code = base
        self.emulated = code >= EMU
        A = torch.empty((m, m), dtype=torch.complex128 if base == 1 else torch.float64, device="cuda")
        B = torch.empty((n, m), dtype=A.dtype, device="cuda")
        st = H.stream_ptr()
        H.hsma_gen_matrix(gen_code, 0, 1, -1, m, m, A.data_ptr(), m, st)
        H.hsma_gen_matrix(gen_code, 1, 1, -1, m, n, B.data_ptr(), m, st)
        if base == 2:
            A, B = A.float(), B.float()
        self.A, self.B, self.B0 = A, B, B.clone()

    def time(self, reps, **cfg):
        H, torch = self.H, self.torch
        opts = H.Opts()
        opts.path = H.PATH_BLOCKED
        opts.fp64_products = 1 if self.emulated else 0
        for k, v in cfg.items():
            setattr(opts, k, v)
        st = H.stream_ptr()

        def run():
            H.hsma_trsm_llnn_ex(self.code, 0, self.m, self.n, 1.0, self.A.data_ptr(), self.m, self.B.data_ptr(),
                                self.m, st, opts=opts)

        run()
        torch.cuda.synchronize()
        best = float("inf")
        for _ in range(reps):
            self.B.copy_(self.B0)
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            e0.record()
            run()
            e1.record()
            torch.cuda.synchronize()
            best = min(best, e0.elapsed_time(e1))
        return best


def key(cfg):
    return ",".join(f"{k}={v}" for k, v in sorted(cfg.items()))


def tune_point(P, code, m, n, reps):
    """Staged search; returns (best configuration, {candidate: ms})."""
    times = {}

    def t(cfg):
        k = key(cfg)
        if k not in times:
            times[k] = P.time(reps, **cfg)
        return times[k]

    if code >= EMU:
        cands = [dict(nb=nb, panel_cols=pc) for nb in EMU_NBS for pc in PANELS]
        best = min(cands, key=t)
        return best, times
    nbs = [nb for nb in NBS if nb <= max(32, 2 * m)]
    best = min((dict(nb=nb) for nb in nbs), key=t)
    if code == 2:
        return best, times
    best = min([best] + [dict(best, tile=tl) for tl in TILES], key=t)
    best = min([best, dict(best, split_k=2)], key=t)
    best = min([best, dict(best, looking=2)], key=t)
    return best, times


def sweep(quick=False, reps=3, budget_s=1800.0):
    import torch
    from paper_2608_25469_gb300 import build as Bld
    Bld.build()
    from paper_2608_25469_gb300 import hsma as H
    grid = QUICK if quick else GRID
    rows, t_start = [], time.time()
    for code, pts in grid.items():
        for (m, n) in pts:
            if time.time() - t_start > budget_s:
                break
            P = Problem(H, torch, code, m, n)
            r = 1 if m * m * n > 4e11 and code < EMU else reps
            best, times = tune_point(P, code, m, n, r)
            full = {"nb": best.get("nb"), "tile": best.get("tile", 0), "split_k": best.get("split_k", 1),
                    "looking": best.get("looking", 1), "panel_cols": best.get("panel_cols", 2048)}
            rows.append({"dtype": code, "m": m, "n": n, **full, "ms": {k: round(v, 4) for k, v in times.items()}})
            print(json.dumps(rows[-1]), flush=True)
            del P
            torch.cuda.empty_cache()
    return rows


NAMES = {0: "HSMA_R64", 1: "HSMA_C128", 2: "HSMA_R32_BF16", EMU + 0: "kEmulatedTableDtype(HSMA_R64)",
         EMU + 1: "kEmulatedTableDtype(HSMA_C128)"}


def write_table(rows, out_dir, data_dir=None):
    inc = ["// Configuration table (dtype, m, n, N_B, tile, split_k, looking, panel_cols): the fastest",
           "// configuration per profiled point on GB300, written by paper_2608_25469_gb300/autotune.py",
           "// (Section 4.3.2's offline profiling); emulated-products entries under dtype + 10.",
           "static const TuneEntry kCompiledTable[] = {"]
    inc += [f"    {{{NAMES[r['dtype']]}, {r['m']}, {r['n']}, {r['nb']}, {r['tile']}, {r['split_k']}, "
            f"{r['looking']}, {r['panel_cols']}}}," for r in rows]
    inc.append("};")
    with open(os.path.join(out_dir, "tuning_table.inc"), "w") as f:
        f.write("\n".join(inc) + "\n")
    data_dir = data_dir or out_dir
    os.makedirs(data_dir, exist_ok=True)
    with open(os.path.join(data_dir, "tuning_gb300.txt"), "w") as f:
        f.write("# dtype m n nb tile split_k looking panel_cols  (fastest per point; every candidate's ms in "
                "tuning_gb300.json; dtype + 10 = emulated FP64 products)\n")
        for r in rows:
            f.write(f"{r['dtype']} {r['m']} {r['n']} {r['nb']} {r['tile']} {r['split_k']} {r['looking']} "
                    f"{r['panel_cols']}\n")
    with open(os.path.join(data_dir, "tuning_gb300.json"), "w") as f:
        json.dump(rows, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out-dir", default=os.path.join(HERE, "csrc"), help="where tuning_table.inc goes")
    ap.add_argument("--data-dir", default=os.path.join(HERE, "tuning"), help="text and JSON copies of the sweep")
    ap.add_argument("--budget-s", type=float, default=1800.0)
    a = ap.parse_args()
    rows = sweep(a.quick, budget_s=a.budget_s)
    os.makedirs(a.out_dir, exist_ok=True)
    write_table(rows, a.out_dir, a.data_dir)


if __name__ == "__main__":
    main()
