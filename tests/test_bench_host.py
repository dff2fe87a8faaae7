"""Host-side logic of bench.py that needs no GPU: the max-over-ranks step time
of the replicated multi-GPU run, exercised with two gloo ranks on CPU."""
import os
import socket

import pytest
import torch.multiprocessing as mp


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    import bench
    out[rank] = bench.max_over_ranks(10.0 + 5.0 * rank, world)
    dist.destroy_process_group()


def test_max_over_ranks_gloo_two_ranks():
    port = _free_port()
    with mp.Manager() as m:
        out = m.dict()
        mp.spawn(_worker, args=(2, port, out), nprocs=2, join=True)
        assert out[0] == 15.0 and out[1] == 15.0


def test_max_over_ranks_single_process():
    import bench
    assert bench.max_over_ranks(3.5, 1) == 3.5


def _run_bench(args, env=None):
    import json
    import os
    import subprocess
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    e = dict(os.environ, **(env or {}))
    r = subprocess.run([sys.executable, os.path.join(root, "bench.py")] + args, cwd=root, env=e,
                       capture_output=True, text=True, timeout=300)
    assert r.returncode == 0, r.stderr[-2000:]
    lines = [l for l in r.stdout.splitlines() if l.startswith("{")]
    return [json.loads(l) for l in lines]


@pytest.mark.parametrize("wx", ["on", "off"])
def test_reference_arm_prints_one_line_on_the_host(wx):
    """The reference arm (the CPU oracle) runs without a GPU and prints one JSON
    line with the contract's keys, on the bench's lists (`--wx-direct`)."""
    out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1",
                      "--ref-sample", "4096", "--wx-direct", wx])
    assert len(out) == 1
    d = out[0]
    assert d["impl"] == "reference" and d["value"] > 0 and d["unit"] == "evals/s"
    assert d["steps"] == 1 and d["warmup"] == 1 and d["higher_is_better"] is True
    assert d["e2e"]["value"] == d["value"] and d["e2e"]["h2d_bytes_per_step"] == 0
    assert d["cpu_baseline"]["kind"] == "oracle" and d["cpu_baseline"]["cores"] >= 1
    assert ("W/X pairs of small leaves direct" in d["config"]["workload"]) == (wx == "on")


def test_reference_arm_other_ranks_exit_quietly():
    out = _run_bench(["--impl", "reference", "--steps", "1", "--warmup", "1",
                      "--ref-sample", "4096"], env={"RANK": "1", "WORLD_SIZE": "2"})
    assert out == []
