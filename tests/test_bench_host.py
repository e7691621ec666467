"""Host-side pieces of bench.py that need no GPU: the replica bookkeeping of the N > 1 path
(run as two gloo ranks on the CPU) and the reference arm's JSON line."""

import json
import os
import socket
import subprocess
import sys

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    sys.path.insert(0, ROOT)
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    t = bench.max_over_ranks(1.5 + rank, "cpu")
    out.put((rank, t, bench.replica_seed(1, rank)))
    dist.barrier()
    dist.destroy_process_group()


def test_replicas_take_the_slowest_rank_and_distinct_seeds():
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    res = sorted(q.get(timeout=120) for _ in procs)
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    assert [t for _, t, _ in res] == [2.5, 2.5]
    assert res[0][2] != res[1][2]


def _run_bench(extra_env=None, *args):
    env = dict(os.environ)
    env.update(extra_env or {})
    r = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference",
                        "--workload", "kicked_ising_L10", "--ref-seconds", "0.2", "--warmup", "0",
                        "--steps", "1", *args], capture_output=True, text=True, env=env,
                       timeout=300)
    return r


def test_reference_arm_prints_one_json_line():
    r = _run_bench()
    assert r.returncode == 0, r.stderr
    lines = [line for line in r.stdout.splitlines() if line.startswith("{")]
    assert len(lines) == 1
    j = json.loads(lines[0])
    for key in ("metric", "value", "unit", "n_gpus", "steps", "warmup", "higher_is_better",
                "config", "cpu_baseline", "e2e"):
        assert key in j
    assert j["impl"] == "reference" and j["higher_is_better"] is False
    assert j["e2e"]["h2d_bytes_per_step"] == 0 and j["cpu_baseline"]["kind"] == "oracle"


def test_reference_arm_non_zero_ranks_exit_quietly():
    r = _run_bench({"WORLD_SIZE": "2", "RANK": "1", "LOCAL_RANK": "1"})
    assert r.returncode == 0
    assert not [line for line in r.stdout.splitlines() if line.startswith("{")]


def test_step_seeds_and_batches():
    sys.path.insert(0, ROOT)
    import bench
    # K steps of rank r solve realisations base + r K + i: distinct within and across ranks
    s0 = bench.step_seeds(1, 0, 20)
    s1 = bench.step_seeds(1, 1, 20)
    assert s0 == list(range(1, 21)) and s1 == list(range(21, 41))
    assert not set(s0) & set(s1)
    # lockstep solves cover every step exactly once, at most `batch` at a time
    for steps, batch in [(20, 2), (7, 2), (5, 4), (1, 2), (3, 1)]:
        b = bench.batches(steps, batch)
        assert sum(b) == steps and max(b) <= batch and min(b) >= 1
    assert bench.batches(0, 2) == []


def test_df_instruction_count_is_the_algorithmic_formula():
    sys.path.insert(0, ROOT)
    import bench
    # two real outputs per amplitude per kicked qubit, 12 FP32 instructions each; one
    # double-float complex product (44) and one complex multiply-add (60) for the Horner
    # epilogue, a second product (44) for the accumulate form
    assert bench.df_instr_per_amplitude(20, "horner") == 24 * 20 + 44 + 60 == 584
    assert bench.df_instr_per_amplitude(16, "acc") == 24 * 16 + 44 + 44 + 60


def test_km_grid_points_are_feasible():
    sys.path.insert(0, ROOT)
    import bench
    for L, nev, k0, m0 in [(20, 100, 16384, 256), (16, 50, 1024, 160), (10, 10, 64, 64),
                           (12, 16, 256, 64)]:
        pts = bench.km_grid(L, nev, k0, m0)
        assert (k0, m0) in pts
        assert len(pts) == len(set(pts))
        for k, m in pts:
            assert 2 <= k <= (1 << L) // 2
            assert nev < m <= min(512, (1 << L) - 1)
            assert m >= min(nev + 16, (1 << L) - 1)
