"""The bench's multi-rank path on CPU: world_size-2 gloo process group on 127.0.0.1.

Ranks are independent replicas (no data-path collective); the only cross-rank steps
are the barrier and the maximum of the timed region over ranks, from which rank 0
reports the whole-job throughput. The reference arm runs on rank 0 only."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank(rank, world, port, results):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank),
                      WORLD_SIZE=str(world))
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        dist.barrier()
        local_ms = 10.0 + 5.0 * rank  # rank 1 is the slow one
        ms = bench.max_over_ranks(local_ms, dist, "cpu")
        results[rank] = (ms, bench.job_rate(world, 100, ms))
        dist.barrier()
    finally:
        dist.destroy_process_group()


def test_two_ranks_report_the_slowest_rank_and_the_whole_job_rate():
    world = 2
    with mp.Manager() as mgr:
        results = mgr.dict()
        mp.start_processes(_rank, args=(world, _free_port(), results), nprocs=world,
                           start_method="spawn", join=True)
        got = dict(results)
    assert set(got) == {0, 1}
    for rank in range(world):
        ms, rate = got[rank]
        assert ms == 15.0  # the maximum over ranks, seen by every rank
        assert rate == pytest.approx(world * 100 / 0.015)


def test_one_process_needs_no_group():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.max_over_ranks(3.5, None, "cpu") == 3.5
    assert bench.job_rate(1, 10, 5.0) == pytest.approx(2000.0)


def test_reference_arm_runs_on_rank_zero_only(capsys):
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_16692_gb300 import workload as W
    # rank 1 of 2 returns at once, before looking at its arguments, timing or printing
    bench.run_reference(None, W.make_params(*W.C1), rank=1, world=2)
    assert capsys.readouterr().out == ""


def test_reference_arm_prints_the_contract_line(capsys):
    """Rank 0 times the oracle and prints one JSON line with the contract's keys; its
    cpu_baseline and e2e carry the line's own value (no transfers)."""
    import json
    import types
    sys.path.insert(0, ROOT)
    import bench
    from paper_2603_16692_gb300 import workload as W
    args = types.SimpleNamespace(steps=2, warmup=1)
    bench.run_reference(args, W.make_params(*W.C1), rank=0, world=1)
    lines = [ln for ln in capsys.readouterr().out.splitlines() if ln.strip()]
    assert len(lines) == 1
    line = json.loads(lines[0])
    for k in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step",
              "higher_is_better", "scaling", "vs_baseline", "dtype", "data", "config",
              "cpu_baseline", "e2e"):
        assert k in line, k
    assert line["impl"] == "reference" and line["value"] > 0 and line["steps"] == 2
    assert line["config"]["workload"].endswith("(2,2^13,7)")
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"]
    assert line["e2e"]["value"] == line["value"]
    assert line["e2e"]["h2d_bytes_per_step"] == line["e2e"]["d2h_bytes_per_step"] == 0


def test_bench_ncu_rows_follow_the_profiled_plan():
    """The roofline's ncu traffic row: the profiled plan's own capture when there is
    one; for the tensor-core-dependent column kernels, the capture with the same kind of
    conversion; nothing for a kernel of an uncaptured plan otherwise."""
    import bench
    r = bench.ncu_row("c3", "DPOB[km4]-tc", "modup_col", True, True)
    assert r["plan"] == "DPOB[km4]-tc" and r["tensor_pct"] > 0
    r = bench.ncu_row("c3", "DPOB[km4]-split-tc", "modup_col", True, True)
    assert r["plan"] == "DPOB[km4]-tc"
    r = bench.ncu_row("c3", "DPOB[km4]-split-tc", "moddown_col", False, False)
    assert r["plan"] == "DPOB[km4,dnr4]-split" and "tensor_pct" not in r
    assert bench.ncu_row("c3", "DPOB[km4]-split-tc", "modup_row_keymult", True, True) is None
    r = bench.ncu_row("c3", "DPOB[km4,dnr4]-split", "modup_row_keymult", False, False)
    assert r["traffic"] > 0
    assert bench.ncu_row("c2", "DPOB-r4", "modup_col", False, False) is None
