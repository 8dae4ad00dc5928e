"""Offline block-size profiling for the blocked path (Section 4.3.2).

For every (dtype, m, n) point of a grid, time the blocked solve for each
candidate diagonal block size N_B, keep the fastest, and write the
"scale x dtype -> block" table: ``csrc/tuning_table.inc`` (compiled into the
library) plus ``tuning/tuning_gb300.txt`` (loadable at run time with
``hsma_tuning_load``) and ``tuning/tuning_gb300.json`` (every candidate's time).  At
run time the planner picks the entry nearest to the input in (log m, log n).

    python -m paper_2608_25469_gb300.autotune [--quick] [--out-dir DIR]

Needs a GPU.  Inputs come from the device-side seeded generator.
"""
from __future__ import annotations

import argparse
import json
import os
import time

HERE = os.path.dirname(os.path.abspath(__file__))
CANDIDATES = (32, 64, 128, 256, 512)

GRID = {
    0: [(m, n) for m in (128, 512, 2048, 8192) for n in (16, 256, 4096)] + [(16384, 16384)],
    1: [(m, n) for m in (128, 512, 2048) for n in (16, 256, 2048)] + [(8192, 8192)],
    2: [(m, n) for m in (128, 512, 2048, 8192) for n in (16, 256, 4096)],
}
QUICK = {0: [(512, 256), (4096, 4096)], 1: [(512, 256), (2048, 2048)], 2: [(1024, 256), (8192, 4096)]}


def time_solve(H, torch, code, m, n, nb, reps):
    import numpy as np  # noqa: F401
    real_dt = {0: torch.float64, 1: torch.complex128, 2: torch.float32}[code]
    gen_code = 1 if code == 1 else 0
    A = torch.empty((m, m), dtype=torch.complex128 if code == 1 else torch.float64, device="cuda")
    B = torch.empty((n, m), dtype=A.dtype, device="cuda")
    st = H.stream_ptr()
    H.hsma_gen_matrix(gen_code, 0, 1, -1, m, m, A.data_ptr(), m, st)
    H.hsma_gen_matrix(gen_code, 1, 1, -1, m, n, B.data_ptr(), m, st)
    if code == 2:
        A = A.to(real_dt)
        B = B.to(real_dt)
    opts = H.Opts()
    opts.path = H.PATH_BLOCKED
    opts.nb = nb
    B0 = B.clone()

    def run():
        H.hsma_trsm_llnn_ex(code, 0, m, n, 1.0, A.data_ptr(), m, B.data_ptr(), m, st, opts=opts)

    run()
    torch.cuda.synchronize()
    best = float("inf")
    for _ in range(reps):
        B.copy_(B0)
        e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
        e0.record()
        run()
        e1.record()
        torch.cuda.synchronize()
        best = min(best, e0.elapsed_time(e1))
    return best


def sweep(quick=False, reps=3, budget_s=900.0):
    import torch
    from paper_2608_25469_gb300 import build as Bld
    Bld.build()
    from paper_2608_25469_gb300 import hsma as H
    grid = QUICK if quick else GRID
    rows, t_start = [], time.time()
    for code, pts in grid.items():
        for (m, n) in pts:
            times = {}
            for nb in CANDIDATES:
                if nb > max(32, 2 * m):
                    continue
                if time.time() - t_start > budget_s:
                    break
                r = 1 if m * m * n > 4e11 else reps
                times[nb] = time_solve(H, torch, code, m, n, nb, r)
            if not times:
                continue
            best = min(times, key=times.get)
            rows.append({"dtype": code, "m": m, "n": n, "nb": best, "ms": {str(k): round(v, 4) for k, v in times.items()}})
            print(json.dumps(rows[-1]), flush=True)
    return rows


def write_table(rows, out_dir, data_dir=None):
    names = {0: "HSMA_R64", 1: "HSMA_C128", 2: "HSMA_R32_BF16"}
    inc = ["// Block-size table (dtype, m, n, N_B): fastest N_B per profiled point on GB300,",
           "// written by paper_2608_25469_gb300/autotune.py (Section 4.3.2's offline profiling).",
           "static const TuneEntry kCompiledTable[] = {"]
    inc += [f"    {{{names[r['dtype']]}, {r['m']}, {r['n']}, {r['nb']}}}," for r in rows]
    inc.append("};")
    with open(os.path.join(out_dir, "tuning_table.inc"), "w") as f:
        f.write("\n".join(inc) + "\n")
    data_dir = data_dir or out_dir
    os.makedirs(data_dir, exist_ok=True)
    with open(os.path.join(data_dir, "tuning_gb300.txt"), "w") as f:
        f.write("# dtype m n nb  (fastest N_B per point; per-candidate ms in tuning_gb300.json)\n")
        for r in rows:
            f.write(f"{r['dtype']} {r['m']} {r['n']} {r['nb']}\n")
    with open(os.path.join(data_dir, "tuning_gb300.json"), "w") as f:
        json.dump(rows, f, indent=1)


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--quick", action="store_true")
    ap.add_argument("--out-dir", default=os.path.join(HERE, "csrc"), help="where tuning_table.inc goes")
    ap.add_argument("--data-dir", default=os.path.join(HERE, "tuning"), help="text and JSON copies of the sweep")
    ap.add_argument("--budget-s", type=float, default=900.0)
    a = ap.parse_args()
    rows = sweep(a.quick, budget_s=a.budget_s)
    os.makedirs(a.out_dir, exist_ok=True)
    write_table(rows, a.out_dir, a.data_dir)


if __name__ == "__main__":
    main()
