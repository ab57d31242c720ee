"""The multi-process path of bench.py on CPU: two gloo ranks, each with its own
timings and edge-update count, must agree on the maximum time and the summed
units (weak scaling: every rank embeds its own instance)."""
import importlib.util
import os
import socket

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, out_dir):
    import torch.distributed as dist
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    spec = importlib.util.spec_from_file_location("bench_dist", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        total, e2e, units = bench.aggregate_over_ranks(10.0 + 5.0 * rank, 20.0 - 3.0 * rank, 1000.0 * (rank + 1),
                                                       "cpu", world)
    finally:
        dist.destroy_process_group()
    with open(os.path.join(out_dir, f"r{rank}.txt"), "w") as f:
        f.write(f"{total} {e2e} {units}\n")


def test_two_gloo_ranks_take_max_time_and_sum_units(tmp_path):
    import torch.multiprocessing as mp
    mp.spawn(_rank_main, args=(2, _free_port(), str(tmp_path)), nprocs=2, join=True)
    for r in range(2):
        total, e2e, units = map(float, open(tmp_path / f"r{r}.txt").read().split())
        assert (total, e2e, units) == (15.0, 20.0, 3000.0)


def test_single_rank_needs_no_process_group():
    spec = importlib.util.spec_from_file_location("bench_single", os.path.join(ROOT, "bench.py"))
    bench = importlib.util.module_from_spec(spec)
    spec.loader.exec_module(bench)
    assert bench.aggregate_over_ranks(12.5, 13.0, 777.0, "cpu", 1) == (12.5, 13.0, 777.0)
