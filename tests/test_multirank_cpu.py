"""Host logic of the multi-rank path, on two gloo ranks on the CPU.

Every rank processes its own configuration (the correlators of different
gauge configurations are independent, so the path shards with no collective on
the data path); the only cross-rank steps are the barriers around the timed
region and the max-over-ranks reduction of its duration.  These tests run that
logic of bench.py on world_size 2 over gloo, and the reference arm under
torchrun, where rank 0 alone works and prints.
"""

import json
import os
import socket
import subprocess
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, outdir):
    sys.path.insert(0, ROOT)
    import bench
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        seed = bench.rank_seed(rank)
        Sl, Ss = bench.make_props_host(2, 1, seed)[0]
        dist.barrier()
        local = 0.25 * (rank + 1)             # rank 1 is the slowest
        ms = bench.max_over_ranks(local, dist, "cpu")
        rate = bench.job_rate(52 * 4, world, ms)
        seeds = [None] * world
        dist.all_gather_object(seeds, (seed, [bench.batched_seed(ci, rank) for ci in range(6)]))
        np.save(os.path.join(outdir, "u%d.npy" % rank), Sl)
        with open(os.path.join(outdir, "r%d.json" % rank), "w") as fh:
            json.dump({"ms": ms, "rate": rate, "seeds": seeds}, fh)
    finally:
        dist.destroy_process_group()


def test_two_gloo_ranks_share_timing_and_own_inputs(tmp_path):
    world = 2
    mp.start_processes(_rank_main, args=(world, free_port(), str(tmp_path)), nprocs=world, start_method="spawn")
    res = [json.load(open(tmp_path / ("r%d.json" % r))) for r in range(world)]
    for r in res:
        assert r["ms"] == 0.5                          # max over ranks, seen by every rank
        assert r["rate"] == pytest.approx(52 * 4 * 2 / 0.5)
    seeds = res[0]["seeds"]
    assert seeds == res[1]["seeds"]
    assert len({s for s, _ in seeds}) == world         # one configuration per rank
    flat = [b for _, bs in seeds for b in bs]
    assert len(set(flat)) == len(flat)                 # batched configurations never repeat across ranks
    u0, u1 = np.load(tmp_path / "u0.npy"), np.load(tmp_path / "u1.npy")
    assert u0.shape == u1.shape and not np.allclose(u0, u1)


def test_reference_arm_under_torchrun_prints_once(tmp_path):
    cmd = [sys.executable, "-m", "torch.distributed.run", "--nnodes=1", "--nproc-per-node", "2",
           "--master-addr", "127.0.0.1", "--master-port", str(free_port()),
           os.path.join(ROOT, "bench.py"), "--impl", "reference", "--gpus", "2", "--steps", "1", "--warmup", "0",
           "--L", "2", "--T", "1"]
    env = dict(os.environ, OMP_NUM_THREADS="1")
    p = subprocess.run(cmd, cwd=ROOT, env=env, capture_output=True, text=True, timeout=300)
    assert p.returncode == 0, p.stderr[-2000:]
    lines = [ln for ln in p.stdout.splitlines() if ln.startswith("{")]
    assert len(lines) == 1
    rec = json.loads(lines[0])
    assert rec["impl"] == "reference" and rec["n_gpus"] == 2 and rec["value"] > 0
    assert rec["e2e"]["h2d_bytes_per_step"] == 0
