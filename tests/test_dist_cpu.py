"""The multi-process host logic of bench.py (one replica per GPU, no data
exchange): two gloo ranks on the CPU.  Each rank solves its own seeds, the
step time is the slowest rank's, the job's throughput counts every rank's
systems, and the reference arm runs on rank 0 alone."""
import json
import os
import socket

import pytest

torch = pytest.importorskip("torch")


def _free_port() -> int:
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, ws, port, out_dir):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(ws),
                      LOCAL_RANK=str(rank))
    import torch.distributed as dist
    dist.init_process_group("gloo", rank=rank, world_size=ws)
    import bench
    res = {"dist": list(bench._dist()),
           "max": bench._max_over_ranks(10.0 + 3.0 * rank, "cpu"),
           "seeds": [s.params["seed"] for s in bench._systems(rank, 3)]}
    bench._oracle_solves = lambda count, start_seed=0: 0.5       # the rank logic, not the oracle, is tested here

    class A:
        steps, warmup, cpu_sample = 2, 1, 4
    ref = bench.run_reference(A)
    res["reference"] = ref
    dist.barrier()
    dist.destroy_process_group()
    with open(os.path.join(out_dir, f"rank{rank}.json"), "w") as f:
        json.dump(res, f)


def test_two_gloo_ranks(tmp_path):
    import torch.multiprocessing as mp
    ws = 2
    mp.spawn(_worker, args=(ws, _free_port(), str(tmp_path)), nprocs=ws, join=True)
    r = [json.load(open(tmp_path / f"rank{k}.json")) for k in range(ws)]
    assert [x["dist"][:2] for x in r] == [[2, 0], [2, 1]]
    assert r[0]["max"] == r[1]["max"] == 13.0                     # the slowest rank's time
    assert r[0]["seeds"] == [0, 1, 2] and r[1]["seeds"] == [3, 4, 5]
    assert r[1]["reference"] is None                             # other ranks exit without work
    ref = r[0]["reference"]
    assert ref["impl"] == "reference" and ref["n_gpus"] == 2
    assert ref["value"] == pytest.approx(2 / 0.5) and ref["e2e"]["h2d_bytes_per_step"] == 0


def test_job_value_counts_every_rank():
    import bench
    assert bench._job_value(4, 608, 500.0) == pytest.approx(4 * 608 / 0.5)
    assert bench._max_over_ranks(7.5, "cpu") == 7.5               # one rank: no collective
