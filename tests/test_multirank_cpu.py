"""Shot-parallel execution across processes, on CPU with gloo (world size 2):
each rank takes its shot range and the FP64 sum of the ranks' gradients and
misfits equals the single-process result. The per-shot gradients here come from
the FP64 oracle (no GPU in this test); on a GPU machine each rank calls sim_adjoint."""
import os
import socket

import numpy as np
import pytest
import torch.multiprocessing as mp

from paper_2605_30541_gb300.shard import shard_shots


def test_shard_ranges_cover_every_shot_once():
    for n in (1, 7, 16, 64):
        for world in (1, 2, 3, 8):
            seen = []
            for r in range(world):
                lo, hi = shard_shots(n, r, world)
                seen += list(range(lo, hi))
            assert seen == list(range(n))


def _case():
    import synth
    c = synth.config_c4(nt=150, nshots=5)
    c.update(nz=40, nx=50)
    c["vel_true"] = synth.procedural_2d(40, 50, 10.0, 4000)
    c["vel"] = synth.smooth(c["vel_true"], 5.0)
    c["src"] = np.stack([np.linspace(50.0, 450.0, 5), np.full(5, 20.0)], axis=1)
    c["rec"] = synth.line(0.0, 490.0, 50, 20.0)
    c["wavelet"] = synth.ricker(15.0, 0.07, 1e-3, 150)
    return c


def _grad(c, shots):
    import oracle
    g = np.zeros(c["vel"].shape)
    J = 0.0
    w = c["wavelet"].astype(np.float64)
    for k in shots:
        d = oracle.forward(c, c["vel_true"].astype(np.float64), w, src=c["src"][k], rec=c["rec"])["gather"]
        o = oracle.gradient(c, c["vel"].astype(np.float64), w, c["src"][k], c["rec"], d)
        g += o["grad"]
        J += o["misfit"]
    return g, J


def _worker(rank, world, port, out):
    import torch
    import torch.distributed as dist
    from paper_2605_30541_gb300.shard import allreduce_fp64, shard_shots
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    c = _case()
    lo, hi = shard_shots(len(c["src"]), rank, world)
    g, J = _grad(c, range(lo, hi))
    gs = allreduce_fp64(torch.from_numpy(g))
    Js = allreduce_fp64(torch.tensor([J]))
    if rank == 0:
        np.save(out, np.concatenate([gs.numpy().ravel(), Js.numpy()]))
    dist.barrier()
    dist.destroy_process_group()


def test_gradient_sum_over_two_gloo_ranks(tmp_path):
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        port = s.getsockname()[1]
    out = str(tmp_path / "sum.npy")
    mp.start_processes(_worker, args=(2, port, out), nprocs=2, start_method="spawn", join=True)
    got = np.load(out)
    c = _case()
    g, J = _grad(c, range(len(c["src"])))
    assert np.allclose(got[:-1], g.ravel(), rtol=1e-12, atol=1e-12 * np.abs(g).max())
    assert abs(got[-1] - J) <= 1e-12 * J
