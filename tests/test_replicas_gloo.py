"""Multi-GPU is replicas only: chains are independent and their random
numbers are keyed by the global chain index, so splitting chains over ranks
and merging the per-rank observables on the host reproduces a single run.
The split is the one bench.py uses: rank r holds the contiguous global
chains r n .. r n + n - 1 and passes chain_offset = r n to the library, whose
Philox key is (seed, chain_offset + local chain).  Checked with two gloo
ranks on the CPU (the oracle sampler stands in for the per-rank GPU work; no
collective is used in the data path, only to gather results and to take the
max of the ranks' times); tests/test_gpu_sampler.py checks on the GPU that
chain_offset reproduces the same chains of a single run."""
import os
import socket

import numpy as np
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import ggf_inputs as gi


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    port = s.getsockname()[1]
    s.close()
    return port


def _chains(p, chain_ids, sweeps, seed):
    from oracle import mcmc, weight
    W = weight.Weights(p)
    out = []
    for c in chain_ids:
        _, obs, _ = mcmc.run_chain(p, W, gi.cold_links(p)[0], seed, c, 0, sweeps)
        out.append(obs)
    return np.array(out)


def _rank(rank, world, port, q):
    os.environ["MASTER_ADDR"] = "127.0.0.1"
    os.environ["MASTER_PORT"] = str(port)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    p = gi.make_problem(2, gi.U1, 1, 2, bond_scale=0.3)
    n = 4 // world
    mine = list(range(rank * n, (rank + 1) * n))                 # global chain ids of this replica
    obs = torch.from_numpy(_chains(p, mine, 3, 99))
    gathered = [torch.zeros_like(obs) for _ in range(world)]
    dist.all_gather(gathered, obs)
    t = torch.tensor([float(rank + 1)], dtype=torch.float64)    # per-rank time: take the max
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    if rank == 0:
        merged = np.zeros((4,) + tuple(obs.shape[1:]))
        n = 4 // world
        for r in range(world):
            merged[r * n:(r + 1) * n] = gathered[r].numpy()
        q.put((merged, float(t[0])))
    dist.barrier()
    dist.destroy_process_group()


def test_two_replicas_merge_to_single_run():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank, args=(r, 2, port, q)) for r in range(2)]
    for pr in procs:
        pr.start()
    merged, tmax = q.get(timeout=300)
    for pr in procs:
        pr.join(timeout=60)
        assert pr.exitcode == 0
    p = gi.make_problem(2, gi.U1, 1, 2, bond_scale=0.3)
    single = _chains(p, range(4), 3, 99)
    assert np.array_equal(merged, single)
    assert tmax == 2.0
