"""Several GPUs, one process each: how the Softmax path shards.

Independent batches (what bench.py --gpus N runs): every rank holds its own batch of m
ciphertexts and its own keys and runs the whole circuit; no data crosses ranks, only the timing
is reduced (the maximum over ranks).

One many-ciphertext Softmax batch split across ranks (Sec. 4.2, Alg. 3): rank r holds a
contiguous share of the m ciphertexts of the main thread.  The only exchange per round is the
auxiliary thread's input S = sum over all m ciphertexts of y (x) y: each rank sums the tensors
of its share, the 3 (level+1) limbs are summed over ranks (one all-reduce of a ciphertext), and
every rank reduces mod q_i and runs the auxiliary thread itself (replicated; cheaper than a
broadcast of lambda).  Residues are below 2^60, so the int64 sum of up to 7 ranks is exact.
"""
from __future__ import annotations


def replica_seeds(rank):
    """Key, input and encryption seeds of an independent replica (distinct per rank)."""
    return {"key": 1234 + rank, "inputs": 100 + rank, "encrypt": 77 + rank}


def max_over_ranks(values, dist=None):
    """Element-wise maximum of a list of floats over all ranks (the job's wall time is the
    slowest rank's); the values themselves when not distributed."""
    if dist is None:
        return [float(v) for v in values]
    import torch

    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend() == "nccl" else torch.device("cpu")
    t = torch.tensor([float(v) for v in values], dtype=torch.float64, device=dev)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return [float(v) for v in t.cpu()]


def shard_range(m, world, rank):
    """Ciphertexts [lo, hi) of a batch of m held by `rank` (contiguous, sizes differ by <= 1)."""
    if not 0 <= rank < world:
        raise ValueError("rank out of range")
    base, extra = divmod(m, world)
    lo = rank * base + min(rank, extra)
    return lo, lo + base + (1 if rank < extra else 0)


MAX_EXACT_RANKS = 7   # 7 (2^60 - 1) < 2^63: the int64 sum of residues cannot overflow


def allreduce_residue_sum(words, dist, group=None):
    """Sums an int64 tensor of residues (each < 2^60) over all ranks in place; the caller
    reduces limb i mod q_i afterwards.  Raises for more ranks than the sum keeps exact."""
    if dist.get_world_size(group) > MAX_EXACT_RANKS:
        raise ValueError("more than %d ranks: reduce partial sums before the all-reduce" % MAX_EXACT_RANKS)
    dist.all_reduce(words, op=dist.ReduceOp.SUM, group=group)
    return words
