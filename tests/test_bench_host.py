"""Host-side logic of bench.py without a GPU: the reduction over ranks of a
multi-GPU run (two gloo ranks on CPU), the per-rank workloads, the oracle
sample of a batch, and the reading of committed ncu summaries."""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)
import bench  # noqa: E402


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    import torch.distributed as dist

    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        # each rank's own replicate: seed = rank, so the workloads differ
        w = bench.make_workloads("room", rank)[0]
        agents = len(w.cells)
        total = bench.max_over_ranks(agents, world, "sum")
        slowest = bench.max_over_ranks(0.5 + rank, world)
        out[rank] = (total, slowest, int(w.cells[:50].sum()))
    finally:
        dist.destroy_process_group()


def test_two_rank_reduction_gloo():
    import torch.multiprocessing as mp

    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(2, port, out), nprocs=2, join=True)
        res = dict(out)
    assert res[0][0] == res[1][0] == 4000.0          # 2 x 2,000 agents, whole job
    assert res[0][1] == res[1][1] == 1.5             # time = max over ranks
    assert res[0][2] != res[1][2]                     # seed + rank: other placements


def test_single_rank_reduction_is_identity():
    assert bench.max_over_ranks(3.5, 1) == 3.5


def test_workload_labels_and_config():
    from paper_0911_2900_gb300 import workloads as wl

    room = [wl.config_small_room(W=60, H=50, n=300, seed=1)]
    assert bench.workload_label(room) == room[0].name
    cfg = bench.workload_config(room, "room")
    assert cfg["agents"] == 300 and cfg["v_m"] == 4
    batch = wl.config_batch(n_rep=3, seed=2, cells_hi=120 ** 2, agents_hi=2000)
    cfg = bench.workload_config(batch, "batch")
    assert cfg["replicates"] == 3
    assert cfg["agents"] == sum(len(w.cells) for w in batch)
    assert sum(cfg["v_m"].values()) == 3


def test_oracle_sample_of_a_batch():
    class W:
        def __init__(self, n):
            self.cells = np.zeros(n, np.int32)

    works = [W(100_000) for _ in range(40)]
    idx = bench.oracle_sample(works, max_agents=1_000_000)
    assert idx == list(range(0, 40, 4))
    assert bench.oracle_sample(works[:5]) == list(range(5))


def test_measured_traffic_follows_the_source_digest(tmp_path):
    d = bench.source_digest("k_plan_direct")
    (tmp_path / "k_plan_direct_wl.md").write_text(
        f"# x\n\nsource_digest: {d}\ndram_bytes_per_launch: 123456\n")
    assert bench.measured_traffic("k_plan_direct", "wl", str(tmp_path)) == 123456.0
    (tmp_path / "k_plan_direct_wl.md").write_text(
        "source_digest: 0000000000000000\ndram_bytes_per_launch: 123456\n")
    assert bench.measured_traffic("k_plan_direct", "wl", str(tmp_path)) is None
    assert bench.measured_traffic("k_plan_direct", "missing", str(tmp_path)) is None


def test_issue_ceiling_from_the_profile(tmp_path, monkeypatch):
    import bench

    p = tmp_path / "k_plan_direct_wl.md"
    p.write_text(f"source_digest: {bench.source_digest('k_plan_direct')}\n"
                 "warp_instructions_per_launch: 1216000\n")
    real = bench.profile_field
    monkeypatch.setattr(bench, "profile_field",
                        lambda k, w, f, d=None: real(k, w, f, str(tmp_path)))
    r = bench.issue_ceiling("k_plan_direct", "wl", 10.0, 2000.0, 152)
    # 1,216,000 / (152 x 4 x 2e9 per s) = 1 us at full issue
    assert abs(r["us_at_full_issue"] - 1.0) < 1e-9 and abs(r["frac_of_issue_peak"] - 0.1) < 1e-9
    assert bench.issue_ceiling("k_plan_direct", "other", 10.0, 2000.0, 152) is None
    assert bench.issue_ceiling("k_plan_direct", "wl", 10.0, None, 152) is None
