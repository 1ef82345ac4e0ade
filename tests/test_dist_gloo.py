"""The multi-GPU path without GPUs: two gloo ranks on the CPU combine their
step times the way bench.py does (the slowest rank sets the job's step time,
the job's rate counts every rank's units), and each rank draws its own
problems (replicas: no data exchange between ranks)."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2410_16727_gb300 import dist as D
from paper_2410_16727_gb300 import inputs as I


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _worker(rank, world, port, out):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        ms_local = 10.0 + 5.0 * rank                 # rank 1 is the slow one
        ms = D.max_over_ranks(ms_local, torch.device("cpu"))
        rate = D.job_throughput(1000.0, ms, world)
        spec = I.WORKLOADS["tiny"]
        cub, _ = I.make_scenes(spec, seed_offset=rank)
        out[rank] = (ms, rate, float(np.asarray(cub[0]).sum()))
    finally:
        dist.destroy_process_group()


def test_two_ranks_combine_like_the_benchmark():
    world = 2
    with mp.get_context("spawn").Manager() as m:      # no fork of this (threaded) process
        out = m.dict()
        mp.start_processes(_worker, args=(world, _free_port(), out), nprocs=world, join=True, start_method="spawn")
        res = dict(out)
    assert res[0][0] == res[1][0] == 15.0                       # max over ranks, seen by both
    assert res[0][1] == res[1][1] == 1000.0 * 2 / 15.0e-3       # units of both ranks / slowest step
    assert res[0][2] != res[1][2]                               # each rank plans its own scenes


def test_single_process_is_the_identity():
    assert D.max_over_ranks(3.5, torch.device("cpu")) == 3.5
    assert D.job_throughput(100.0, 2.0, 1) == 100.0 / 2.0e-3
