"""Host-side logic of the multi-GPU bench path (no GPU): with --gpus N every
rank runs an independent replica; the whole-job value is the points of all
ranks over the slowest rank's time.  Two gloo ranks on CPU exercise the
all-reduce; the reference arm's other ranks exit without work."""
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, ws, port, q):
    import torch.distributed as dist
    os.environ.update({"MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port), "RANK": str(rank),
                       "WORLD_SIZE": str(ws), "LOCAL_RANK": str(rank)})
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    try:
        # rank r timed its 4 steps in (100 + 50 r) ms
        ms, value = bench.aggregate_replicas(100.0 + 50.0 * rank, 4, 1_000_000, ws, "cpu")
        q.put((rank, ms, value, bench._dist()))
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_take_the_slowest_rank_and_count_all_points():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(timeout=120)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(2))
    for rank, ms, value, dist_env in got:
        assert dist_env == (2, rank, rank)
        assert ms == pytest.approx(150.0 / 4)              # the slower rank: 150 ms over 4 steps
        assert value == pytest.approx(2 * 1_000_000 / (150.0 / 4 / 1e3))


def test_single_rank_needs_no_process_group():
    sys.path.insert(0, ROOT)
    import bench
    ms, value = bench.aggregate_replicas(80.0, 8, 500, 1)
    assert ms == pytest.approx(10.0) and value == pytest.approx(500 / 0.010)


def test_reference_arm_other_ranks_exit_without_work(monkeypatch):
    sys.path.insert(0, ROOT)
    import bench
    monkeypatch.setenv("WORLD_SIZE", "2")
    monkeypatch.setenv("RANK", "1")
    monkeypatch.setenv("LOCAL_RANK", "1")
    args = bench._args([])
    assert bench.run_reference(args) == 0


def test_reference_arm_line_keeps_the_contract(monkeypatch, capsys):
    """Rank 0 of the reference arm prints one JSON line with the base keys,
    impl "reference", a cpu_baseline describing the run and an e2e with no
    host-device bytes (a small N keeps this to a second or two)."""
    import json
    sys.path.insert(0, ROOT)
    import bench
    for k in ("WORLD_SIZE", "RANK", "LOCAL_RANK"):
        monkeypatch.delenv(k, raising=False)
    assert bench.run_reference(bench._args(["--impl", "reference", "--n", "3000", "--steps", "1",
                                            "--warmup", "0"])) == 0
    line = json.loads(capsys.readouterr().out.strip().splitlines()[-1])
    for k in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
              "scaling", "vs_baseline", "dtype", "data", "config"):
        assert k in line, k
    assert line["impl"] == "reference" and line["steps"] == 1 and line["value"] > 0
    assert line["unit"] == bench.UNIT and line["metric"] == bench.METRIC and line["higher_is_better"] is True
    assert line["config"]["workload"] == bench.WORKLOAD
    cb = line["cpu_baseline"]
    assert cb["kind"] == "oracle" and cb["cores"] >= 1 and cb["value"] == line["value"] and cb["sample"]
    assert line["e2e"] == {"value": line["value"], "unit": line["unit"], "h2d_bytes_per_step": 0,
                           "d2h_bytes_per_step": 0}
