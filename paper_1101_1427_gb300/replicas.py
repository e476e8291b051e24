"""Partitioning of independent work over processes (one per GPU).

Realisations of a disordered system, lattices at different temperatures and
whole replicas are independent, so N GPUs run disjoint shards with no
exchange on the data path (weak scaling); only timing and bookkeeping use the
process group.  Random words are keyed by global indices, so a shard draws
exactly the numbers the same units would draw in an unsharded run.
"""


def shard(n_units, world, rank):
    """Contiguous, balanced share [start, stop) of n_units for `rank`."""
    if world < 1 or not 0 <= rank < world or n_units < 0:
        raise ValueError("bad shard request")
    base, extra = divmod(n_units, world)
    start = rank * base + min(rank, extra)
    return start, start + base + (1 if rank < extra else 0)


def shard_groups(n_real, world, rank, group=32):
    """Share of realisation groups of `group` realisations (multi-spin coding
    packs 32 realisations per word, so shards never split a group)."""
    g0, g1 = shard(n_real // group, world, rank)
    return g0 * group, g1 * group
