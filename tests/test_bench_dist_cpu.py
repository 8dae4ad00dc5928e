"""bench.py's multi-rank host logic on CPU: gloo, world size 2 (no GPU)."""
import json
import os
import subprocess
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _worker(rank, world, port, out):
    os.environ.update(RANK=str(rank), WORLD_SIZE=str(world), LOCAL_RANK=str(rank), MASTER_ADDR="127.0.0.1",
                      MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    d = bench.Dist()
    d.init("gloo")
    t_max = d.max(float(rank + 1) * 10.0)
    f_sum = d.sum(1.5 * (rank + 1))
    d.barrier()
    out[rank] = (t_max, f_sum, bench.shard_seed(7, rank))
    d.close()


def test_two_ranks_max_time_and_total_work():
    world, port = 2, 29517
    mgr = mp.Manager()
    out = mgr.dict()
    ctx = mp.get_context("spawn")
    ps = [ctx.Process(target=_worker, args=(r, world, port, out)) for r in range(world)]
    [p.start() for p in ps]
    [p.join(120) for p in ps]
    assert all(p.exitcode == 0 for p in ps)
    assert out[0][0] == out[1][0] == 20.0        # max over ranks of the timed region
    assert out[0][1] == out[1][1] == 4.5         # whole-job work is the sum over ranks
    assert out[0][2] != out[1][2]                # each rank solves its own batch


def test_reference_arm_nonzero_rank_exits_quietly():
    env = dict(os.environ, RANK="1", WORLD_SIZE="2", LOCAL_RANK="1")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=300)
    assert r.returncode == 0 and r.stdout.strip() == ""


def test_reference_arm_rank0_line():
    env = dict(os.environ, RANK="0", WORLD_SIZE="1", LOCAL_RANK="0")
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--steps", "1",
                        "--warmup", "3"], env=env, capture_output=True, text=True, timeout=600)
    assert r.returncode == 0, r.stderr
    line = json.loads(r.stdout.strip().splitlines()[-1])
    assert line["impl"] == "reference" and line["unit"] == "GFLOP/s" and line["value"] > 0
    assert line["cpu_baseline"]["kind"] == "oracle" and line["e2e"]["h2d_bytes_per_step"] == 0


def test_bench_emulated_panel_width_matches_library():
    """bench.py counts the emulated update work with the panel width the plan reports,
    and its fallback is the library's default width."""
    import re
    sys.path.insert(0, ROOT)
    import bench
    src = open(os.path.join(ROOT, "paper_2608_25469_gb300", "csrc", "mixed.h")).read()
    lib = int(re.search(r"kEmuPanelColsDefault = (\d+);", src).group(1))
    assert bench.EMU_PANEL_COLS == lib
    assert "info.plan.panel_cols" in open(os.path.join(ROOT, "bench.py")).read()


def test_profile_traffic_follows_source_hash_and_scales_by_work(tmp_path, monkeypatch):
    """A committed ncu summary's DRAM bytes are used only while the hash of the kernel's
    sources matches, and are scaled by the bench launch's work when the capture was smaller."""
    sys.path.insert(0, ROOT)
    import bench
    src = tmp_path / "k.cu"
    src.write_text("kernel v1\n")
    (tmp_path / "profiles").mkdir()
    monkeypatch.setattr(bench, "ROOT", str(tmp_path))
    sha = bench.source_sha(["k.cu"])
    (tmp_path / "profiles" / "p.txt").write_text(
        f"# title\nsource_sha256_16: {sha}\ndram_bytes_per_launch: 1000\nwork_per_launch: 10\n")
    assert bench.profile_traffic("p.txt", ["k.cu"]) == 1000.0
    assert bench.profile_traffic("p.txt", ["k.cu"], work=25) == 2500.0
    src.write_text("kernel v2\n")  # the kernel changed since the capture
    assert bench.profile_traffic("p.txt", ["k.cu"]) is None
    assert bench.profile_traffic("missing.txt", ["k.cu"]) is None


def test_committed_profiles_are_well_formed():
    """Every summary under profiles/ gives the ncu command that made it, the sources it was
    taken on (which exist) and their hash; a hash that no longer matches (the kernel changed
    since the capture, so the bench reports no traffic figure) is reported as a warning."""
    import warnings
    sys.path.insert(0, ROOT)
    import bench
    names = sorted(os.listdir(os.path.join(ROOT, "profiles")))
    assert names
    for name in names:
        kv = {}
        for line in open(os.path.join(ROOT, "profiles", name)):
            if ":" in line:
                k, v = line.split(":", 1)
                kv.setdefault(k.strip(), v.strip())
        assert kv["command"].startswith("ncu ") and "--clock-control none" in kv["command"], name
        files = [x.strip() for x in kv["sources"].split(",")]
        assert all(os.path.exists(os.path.join(ROOT, f)) for f in files), name
        float(kv["dram_bytes_per_launch"])
        if kv["source_sha256_16"] != bench.source_sha(files):
            warnings.warn(f"profiles/{name} was captured on older sources")
