"""The multi-rank paths on CPU ranks (torch.distributed, gloo, world size 2).

1. Independent replicas (bench.py --gpus N): distinct seeds per rank, the job time is the
   maximum over ranks on every rank.
2. One many-ciphertext batch split across ranks (the exchange step of Alg. 3): each rank sums
   y (x) y over its share of the m ciphertexts with the oracle, the partial tensors are summed by
   one all-reduce and reduced mod q_i, and the relinearised S equals the unsplit computation
   limb for limb on both ranks."""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _init(rank, world, port):
    for p in (ROOT, os.path.join(ROOT, "oracle")):
        if p not in sys.path:
            sys.path.insert(0, p)
    dist.init_process_group("gloo", init_method="tcp://127.0.0.1:%d" % port, rank=rank, world_size=world)


def _replicas(rank, world, port):
    _init(rank, world, port)
    from paper_2410_11184_gb300 import shard

    seeds = [None] * world
    dist.all_gather_object(seeds, shard.replica_seeds(rank))
    assert len({tuple(sorted(s.items())) for s in seeds}) == world   # no two replicas share a seed
    ms = shard.max_over_ranks([100.0 + rank, 50.0 - rank], dist)
    assert ms == [100.0 + world - 1, 50.0]
    dist.destroy_process_group()


def _split_square_sum(rank, world, port):
    _init(rank, world, port)
    import oracle as O
    from paper_2410_11184_gb300 import he, shard

    chains, _, _ = he.load_params()
    ch = chains["toy"]
    o = O.Oracle(ch)
    o.keygen(7)
    m, level = 5, 6
    rng = np.random.default_rng(3)
    cts = [o.encrypt(rng.uniform(-1, 1, o.n0), level, 2.0 ** 40, 11, i) for i in range(m)]
    q = np.array(o.q[:level + 1], dtype=object)

    def tensor_sum(idx):
        acc = np.zeros((3, level + 1, o.n), dtype=object)
        for i in idx:
            acc = acc + o.tensor(cts[i], cts[i]).astype(object)
        return (acc % q[None, :, None]).astype(np.uint64)

    lo, hi = shard.shard_range(m, world, rank)
    part = torch.from_numpy(tensor_sum(range(lo, hi)).astype(np.int64))
    shard.allreduce_residue_sum(part, dist)
    summed = (part.numpy().astype(object) % q[None, :, None]).astype(np.uint64)
    s_split = o.relin(summed, level)
    s_whole = o.relin(tensor_sum(range(m)), level)
    assert np.array_equal(s_split, s_whole)
    # the auxiliary thread then runs on identical inputs on every rank
    both = [None] * world
    dist.all_gather_object(both, s_split.tobytes())
    assert all(b == both[0] for b in both)
    dist.destroy_process_group()


@pytest.mark.parametrize("fn", [_replicas, _split_square_sum])
def test_two_cpu_ranks(fn):
    mp.spawn(fn, args=(2, _free_port()), nprocs=2, join=True)


def test_shard_range_partitions():
    from paper_2410_11184_gb300 import shard

    for m in (1, 5, 64):
        for world in (1, 2, 3, 8):
            parts = [shard.shard_range(m, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == m
            assert all(a[1] == b[0] for a, b in zip(parts, parts[1:]))
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
