"""The multi-rank host logic of bench.py (weak scaling over independent pairs), run as two
`gloo` ranks on CPU: the job time is the slowest rank's, the value counts every rank's pairs,
each rank draws its own pair, and the reference arm runs on rank 0 only."""
import json
import os
import socket
import sys

import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
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
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seconds = [1.5, 2.5][rank]
        slowest = bench.max_over_ranks(seconds, dist, "cpu")
        pairs_per_rank = 3
        out[rank] = (slowest, world * pairs_per_rank / slowest, bench.rank_seed(7, rank))
    finally:
        dist.destroy_process_group()


def test_weak_scaling_aggregation_over_two_gloo_ranks():
    world = 2
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_rank_main, args=(world, _free_port(), out), nprocs=world, join=True)
        res = dict(out)
    # both ranks agree on the slowest rank's time and on the whole-job value
    assert res[0][0] == res[1][0] == 2.5
    assert res[0][1] == res[1][1] == pytest.approx(2 * 3 / 2.5)
    # independent pairs: every rank its own seed
    assert res[0][2] != res[1][2]


def test_single_rank_needs_no_process_group():
    import bench
    assert bench.max_over_ranks(1.25) == 1.25
    assert bench.rank_seed(7, 0) == 7


def test_reference_arm_prints_on_rank_zero_only(capsys):
    import bench
    args = bench.argparse.Namespace(workload="fp64_small", steps=1, warmup=0, pairs=4, holdout=4)
    bench.run_reference(args, rank=1, world=2)
    assert capsys.readouterr().out == ""


@pytest.mark.parametrize("workload", ["fp64_small", "batched"])
def test_reference_arm_json_line_contract(workload):
    # bench.py --impl reference on the host cores (the oracle): one JSON line with the contract's keys;
    # the batched workload (the default) solves one pair of the batch per step
    import subprocess
    extra = ["--pairs", "2"] if workload == "batched" else []
    out = subprocess.run([sys.executable, os.path.join(ROOT, "bench.py"), "--impl", "reference", "--workload",
                          workload, "--steps", "1", "--warmup", "0", *extra], capture_output=True, text=True,
                         timeout=300, cwd=ROOT)
    assert out.returncode == 0, out.stderr[-2000:]
    lines = [ln for ln in out.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    d = json.loads(lines[0])
    for key in ("impl", "metric", "value", "unit", "n_gpus", "steps", "warmup", "ms_per_step", "higher_is_better",
                "scaling", "vs_baseline", "dtype", "data", "config", "cpu_baseline", "e2e"):
        assert key in d, key
    assert d["impl"] == "reference" and d["value"] > 0 and d["cpu_baseline"]["kind"] == "oracle"
    assert d["e2e"]["h2d_bytes_per_step"] == 0 and d["e2e"]["value"] == d["value"]
    assert d["steps"] == 1 and d["warmup"] == 3
