"""The bench's multi-rank timing path on CPU ranks (gloo, world size 2).

Every rank times its own replica; the job's step time is the slowest rank's,
and the throughput counts the units of all ranks.  The reference arm runs on
rank 0 only.
"""

import os
import socket

import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import bench


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        bench.rank_barrier(world, dist)
        local_ms = 10.0 * (rank + 1)  # the last rank is the slowest
        t = bench.max_over_ranks(local_ms, world, dist, torch.device("cpu"))
        q.put((rank, t, bench.whole_job_rate(60000, t, world)))
        bench.rank_barrier(world, dist)
    finally:
        dist.destroy_process_group()


def test_two_ranks_take_the_slowest_rank_and_count_all_units():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(2))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r for r, _, _ in res] == [0, 1]
    for _, t, rate in res:
        assert t == 20.0
        assert abs(rate - 2 * 60000 / 0.020) < 1e-6


def test_single_rank_helpers_need_no_process_group():
    assert bench.max_over_ranks(3.5, 1, None, torch.device("cpu")) == 3.5
    bench.rank_barrier(1, None)
    assert bench.whole_job_rate(1000, 500.0, 1) == 2000.0


def test_reference_arm_runs_on_rank_zero_only(capsys):
    class Args:
        workload, warmup, steps = "water10k", 0, 0
    assert bench.run_reference(Args(), rank=1, world=2) is None
    assert capsys.readouterr().out == ""


def test_csc_asymmetry_of_a_collected_matrix():
    # column-collected D: column j carries its own subgraph's rows, so
    # D_jk and D_kj come from different subgraphs (or one is absent)
    import numpy as np
    rng = np.random.default_rng(3)
    n = 7
    a = rng.normal(size=(n, n))
    s = a + a.T
    s[np.abs(s) < 0.5] = 0.0
    import scipy.sparse as sp
    m = sp.csc_matrix(s)
    assert bench.csc_asymmetry(n, m.indptr, m.indices, m.data) == 0.0
    t = s.copy()
    t[1, 4] += 0.25          # one entry perturbed
    t[5, 2], t[2, 5] = 0.75, 0.0   # one side absent
    m2 = sp.csc_matrix(t)
    assert abs(bench.csc_asymmetry(n, m2.indptr, m2.indices, m2.data) - max(0.25, 0.75)) < 1e-15


def test_trajectory_mu_start_extrapolates_consecutive_geometries():
    import math
    import bench
    assert math.isnan(bench.extrapolated_mu([], 0))
    assert bench.extrapolated_mu([(0, -7.5)], 1) == -7.5
    assert bench.extrapolated_mu([(0, -7.5), (1, -7.4)], 2) == 2.0 * -7.4 - -7.5
    # a jump in the geometry sequence (the timed steps restart at geometry 0)
    assert bench.extrapolated_mu([(1, -7.4), (2, -7.3)], 0) == -7.3


def test_recorded_traffic_only_for_the_sources_it_was_taken_on(tmp_path, monkeypatch):
    # the roofline's DRAM traffic comes from a recorded ncu capture only while
    # the recursion kernel's sources still hash to what the record names
    import json
    rec = {"kernel": "k_fermi_split", "traffic_bytes_per_launch": 123456789}
    path = tmp_path / "traffic.json"
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(path))
    path.write_text(json.dumps(dict(rec, kernel_source_sha256=bench.kernel_source_hash())))
    assert bench.recorded_traffic() == 123456789.0
    path.write_text(json.dumps(dict(rec, kernel_source_sha256="0" * 64)))
    assert bench.recorded_traffic() is None
    monkeypatch.setattr(bench, "TRAFFIC_FILE", str(tmp_path / "missing.json"))
    assert bench.recorded_traffic() is None
