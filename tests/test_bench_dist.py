"""The benchmark's multi-rank path on the CPU: world size 2 over gloo.

bench.py runs one independent replica per rank (no collective on the data
path); the ranks only meet at the barriers around the timed region and in the
maximum of their durations, and rank 0 alone prints.  These tests run that
coordination (bench.Ranks, whole_job_rate) in two gloo processes, and the
reference arm (the FP64 oracle on a bounded sample) under torchrun with two
ranks."""
import json
import os
import socket
import subprocess
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    import bench
    ranks = bench.Ranks(world, rank, backend="gloo")
    ranks.barrier()
    # each replica "took" a different time; the job's time is the slowest rank's
    mine = 0.010 * (rank + 1)
    slowest = ranks.max_over_ranks(mine)
    rate = bench.whole_job_rate(world, 50, 1 << 24, slowest)
    ranks.barrier()
    out.put((rank, ranks.root, mine, slowest, rate))
    ranks.close()


def test_two_gloo_ranks_barrier_max_and_rate():
    world, port = 2, _free_port()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in range(world))
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [r[1] for r in res] == [True, False]          # rank 0 is the root
    assert all(r[3] == pytest.approx(0.020) for r in res)  # max over ranks on every rank
    # whole-job aggregate: both ranks' samples over the slowest rank's time
    assert res[0][4] == pytest.approx(2 * 50 * (1 << 24) / 0.020 / 1e9)
    assert res[0][4] == res[1][4]


def test_single_process_ranks_are_no_ops():
    import bench
    r = bench.Ranks(1, 0)
    r.barrier()
    assert r.root and r.max_over_ranks(1.5) == 1.5
    assert bench.whole_job_rate(1, 10, 1000, 2.0) == pytest.approx(10 * 1000 / 2.0 / 1e9)
    r.close()


def test_reference_arm_under_torchrun_prints_once():
    """`bench.py --impl reference` with two ranks: rank 0 times the oracle and
    prints one JSON line; the other rank exits 0 without work."""
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(_free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "2", "--warmup", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="2")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=600)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1, p.stdout
    d = json.loads(lines[0])
    assert d["impl"] == "reference" and d["n_gpus"] == 2 and d["steps"] == 2
    assert d["cpu_baseline"]["kind"] == "oracle" and d["value"] > 0
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["d2h_bytes_per_step"] == 0


def test_oracle_timing_of_every_workload():
    """bench.cpu_oracle_configs (the cpu_baseline's all_workloads object) on two
    threads: every workload timed with all and with one thread."""
    import bench
    out = bench.cpu_oracle_configs(2)
    assert out["kind"] == "oracle" and out["threads_multi"] == 2
    names = {"cfg0_2p16_P5M2", "cfg1_2p24_P9M4", "cfg2_batched_64", "cfg3_fwd_grad_P7M3", "cfg4_ls_P11M7"}
    assert set(out["configs"]) == names
    for c in out["configs"].values():
        assert c["multi"] > 0 and c["single_thread"] > 0 and c["sample"] and c["unit"]
