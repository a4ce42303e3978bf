"""The multi-GPU benchmark path on CPU: world_size-2 gloo ranks (no GPU). Independent problems
shard across ranks with no data-path collective; each rank draws its own seeds, and the
weak-scaling time is the maximum over ranks."""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
dist = pytest.importorskip("torch.distributed")


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _rank_main(rank, world, port, out):
    import sys
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    sys.path.insert(0, root)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as d

    import bench
    d.init_process_group("gloo", rank=rank, world_size=world)
    w = dict(bench.WORKLOADS["c2"], batch=3, n=16)
    u0 = bench.u0_batch(w, rank)
    # each rank's own problem seeds: rank r takes seeds r * batch .. r * batch + batch - 1
    seeds = [rank * w["batch"] + b for b in range(w["batch"])]
    t = bench.max_over_ranks(10.0 * (rank + 1), d, torch.device("cpu"))
    gathered = [torch.zeros(u0.size, dtype=torch.float64) for _ in range(world)]
    d.all_gather(gathered, torch.from_numpy(u0.ravel()))
    if rank == 0:
        np.save(out, np.stack([g.numpy() for g in gathered]))
        with open(out + ".txt", "w") as f:
            f.write(f"{t} {seeds}\n")
    d.barrier()
    d.destroy_process_group()


def test_two_ranks_draw_disjoint_seeds_and_report_the_slowest_time(tmp_path):
    import torch.multiprocessing as mp

    import ch_inputs
    out = str(tmp_path / "u0.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), out), nprocs=2, start_method="spawn")
    u = np.load(out)
    n, batch = 16, 3
    for r in range(2):
        want = np.stack([ch_inputs.initial_condition(1, n, r * batch + b, amp=0.1) for b in range(batch)])
        assert np.array_equal(u[r].reshape(batch, n), want)
    assert not np.array_equal(u[0], u[1])
    t = float(open(out + ".txt").read().split()[0])
    assert t == 20.0  # max over ranks of 10 (rank + 1)
