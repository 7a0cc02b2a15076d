"""Multi-process paths on CPU ranks (gloo, world size 2, no GPU).

* The benchmark's distributed plumbing: process-group setup from the
  launcher's environment, the barrier, and the max / sum reductions that turn
  per-rank times and units into the job's figures.
* The sharded combine of one image over several ranks: each rank holds a
  contiguous part of the pixels, computes its memberships (Eq. 4) and its
  FP64 partial sums of Eq. 3 and Eq. 1 and its max |dU|, and one all-reduce
  per iteration (sum, and max for the stopping quantity) gives every rank the
  same V^{k+1} and the same decision. The result must equal the unsharded
  FP64 oracle run (Algorithm 1) on the whole image.
"""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

import oracle
import phantom


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _env(rank, world, port):
    os.environ.update({"RANK": str(rank), "WORLD_SIZE": str(world), "LOCAL_RANK": str(rank),
                       "MASTER_ADDR": "127.0.0.1", "MASTER_PORT": str(port)})


def _bench_worker(rank, world, port, out):
    import sys
    sys.path.insert(0, os.path.dirname(os.path.dirname(os.path.abspath(__file__))))
    _env(rank, world, port)
    import torch.distributed as dist
    import bench
    w, r, _ = bench.dist_setup()
    assert (w, r) == (world, rank)
    bench.barrier(w)
    mx = bench.allreduce(float(rank + 1) * 1.5, "max", w)
    sm = bench.allreduce(float(rank + 1), "sum", w)
    out[rank] = (mx, sm, dist.get_backend())
    dist.destroy_process_group()


def test_bench_reductions_over_two_gloo_ranks():
    world, port = 2, _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_bench_worker, args=(world, port, out), nprocs=world, join=True)
    for r in range(world):
        assert out[r] == (3.0, 3.0, "gloo")


def _sharded_worker(rank, world, port, x, u0, C, m, eps, max_iter, out):
    import torch
    import torch.distributed as dist
    _env(rank, world, port)
    dist.init_process_group("gloo")
    n = x.size
    lo, hi = rank * n // world, (rank + 1) * n // world
    xs, us = x[lo:hi], u0[:, lo:hi]
    # pass 0: V^1 from U^0 (Eq. 3), partial sums all-reduced in FP64
    w = us ** m
    t = torch.tensor(np.concatenate([w @ xs, w.sum(1)]), dtype=torch.float64)
    dist.all_reduce(t)
    V = (t[:C] / t[C:]).numpy()
    Uprev = us
    k, status = 0, "not converged"
    for k in range(1, max_iter + 1):
        U = oracle.memberships(xs, V, m)                   # Eq. 4 on this rank's pixels
        d = torch.tensor([np.max(np.abs(U - Uprev))], dtype=torch.float64)
        w = U ** m
        J = np.sum(w * (xs[None, :] - V[:, None]) ** 2)    # Eq. 1, this rank's part
        s = torch.tensor(np.concatenate([w @ xs, w.sum(1), [J]]), dtype=torch.float64)
        dist.all_reduce(s)
        dist.all_reduce(d, op=dist.ReduceOp.MAX)
        if d.item() < eps:
            status = "converged"
            break
        V = (s[:C] / s[C:2 * C]).numpy()
        Uprev = U
    out[rank] = (V.copy(), k, status, float(s[2 * C]))
    dist.destroy_process_group()


@pytest.mark.parametrize("world", [2, 3])
def test_sharded_combine_equals_the_unsharded_oracle(world):
    img, _ = phantom.phantom2d(7, 48, 40, 8.0)
    x = img.reshape(-1).astype(np.float64)
    C, m, eps, max_iter = 4, 2.0, 1e-9, 200
    u0 = phantom.dirichlet_u0((7, 2), C, x.size).astype(np.float64)
    ref = oracle.fcm(x, C, m, eps, max_iter, U0=u0, want_U=False)
    port = _free_port()
    out = mp.get_context("spawn").Manager().dict()
    mp.spawn(_sharded_worker, args=(world, port, x, u0, C, m, eps, max_iter, out), nprocs=world, join=True)
    for r in range(world):
        V, k, status, J = out[r]
        assert k == ref["iters"] and status == "converged"
        assert np.max(np.abs(V - ref["V"]) / np.maximum(np.abs(ref["V"]), 1.0)) <= 1e-12
        assert abs(J - ref["J"][-1]) <= 1e-10 * abs(ref["J"][-1])
    # every rank took the same decisions and holds the same centers
    assert all(np.array_equal(out[0][0], out[r][0]) for r in range(world))
