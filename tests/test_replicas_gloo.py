"""The multi-GPU path of bench.py is N independent replicas (no data-path
collective): its rank bookkeeping and the whole-job aggregation (slowest rank's
time, all ranks' work) run here as world-size-2 gloo process groups on CPU."""
import json
import os
import socket
import sys

import pytest
import torch.multiprocessing as mp

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import torch.distributed as dist
    import bench
    dist.init_process_group("gloo", rank=rank, world_size=world)
    r, lr, w = bench.dist_env()
    secs, units = bench.aggregate(dist, 1.0 + 0.5 * rank, 1000.0 * (rank + 1), "cpu")
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(outdir, f"r{rank}.json"), "w") as f:
        json.dump({"rank": r, "local": lr, "world": w, "secs": secs, "units": units}, f)


def test_replica_aggregation_world2(tmp_path):
    port = _free_port()
    mp.start_processes(_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    for rank in range(2):
        with open(tmp_path / f"r{rank}.json") as f:
            r = json.load(f)
        assert (r["rank"], r["local"], r["world"]) == (rank, rank, 2)
        assert r["secs"] == pytest.approx(1.5)          # the slowest rank
        assert r["units"] == pytest.approx(3000.0)      # all ranks' work


def test_single_process_aggregation_is_identity():
    sys.path.insert(0, ROOT)
    import bench
    assert bench.aggregate(None, 2.5, 7.0, "cpu") == (2.5, 7.0)


def _ref_worker(rank, world, port, outdir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), LOCAL_RANK=str(rank),
                      WORLD_SIZE=str(world))
    sys.path.insert(0, ROOT)
    import argparse
    import io
    import contextlib
    import bench
    args = argparse.Namespace(workload="bmatch-2k", steps=1, warmup=0, step=None, gpus=world, cpu_procs=2)
    buf = io.StringIO()
    with contextlib.redirect_stdout(buf):
        bench.run_reference(args)
    with open(os.path.join(outdir, f"ref{rank}.txt"), "w") as f:
        f.write(buf.getvalue())


def test_reference_arm_prints_on_rank0_only(tmp_path):
    """Under torchrun only rank 0 runs the oracle arm and prints its line."""
    port = _free_port()
    mp.start_processes(_ref_worker, args=(2, port, str(tmp_path)), nprocs=2, join=True, start_method="spawn")
    out0 = (tmp_path / "ref0.txt").read_text().strip().splitlines()
    out1 = (tmp_path / "ref1.txt").read_text().strip()
    assert out1 == ""
    line = json.loads(out0[-1])
    assert line["impl"] == "reference" and line["value"] > 0 and line["e2e"]["h2d_bytes_per_step"] == 0
