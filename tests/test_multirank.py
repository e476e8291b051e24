"""Multi-process path on the CPU (gloo, world size 2): work is sharded over
ranks with no data-path exchange, and the union of the shards equals the
unsharded computation (the oracle stands in for each rank's GPU work)."""
import os
import socket

import numpy as np
import pytest

from paper_1101_1427_gb300.replicas import shard, shard_groups


def test_shard_partitions_exactly():
    for n in (0, 1, 5, 32, 1024, 1025):
        for world in (1, 2, 3, 8):
            parts = [shard(n, world, r) for r in range(world)]
            assert parts[0][0] == 0 and parts[-1][1] == n
            for (a, b), (c, d) in zip(parts, parts[1:]):
                assert b == c and a <= b
            sizes = [b - a for a, b in parts]
            assert max(sizes) - min(sizes) <= 1
    assert shard_groups(1024, 2, 1) == (512, 1024)
    with pytest.raises(ValueError):
        shard(4, 2, 2)


def _free_port():
    s = socket.socket()
    s.bind(("127.0.0.1", 0))
    p = s.getsockname()[1]
    s.close()
    return p


def _rank_main(rank, world, port, reals, out_path):
    import torch.distributed as dist
    import oracle
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    L, seed, n, betas = 4, 9, 6, [0.9, 1.4, 2.0]
    a, b = shard(len(reals), world, rank)
    rows = []
    for r in reals[a:b]:
        J = oracle.ea_couplings(3, L, r, seed)
        s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(k, r >> 5, t), bit=r & 31)
                                for t in range(3)]) for k in range(2)]).copy()
        E, Q, acc, _ = oracle.pt_run(3, L, s, betas, seed, r, r >> 5, 0, n, 1, J=J)
        rows.append(np.concatenate([E.ravel(), Q.ravel(), s.ravel().astype(np.int64)]))
    gathered = [None] * world
    dist.all_gather_object(gathered, np.stack(rows))
    if rank == 0:
        np.save(out_path, np.concatenate(gathered))
    dist.barrier()
    dist.destroy_process_group()


def test_two_gloo_ranks_equal_unsharded(tmp_path):
    import torch.multiprocessing as mp
    import oracle
    reals = [0, 5, 31, 32, 40, 63]
    out = str(tmp_path / "gathered.npy")
    mp.start_processes(_rank_main, args=(2, _free_port(), reals, out), nprocs=2, join=True,
                       start_method="spawn")
    got = np.load(out)
    L, seed, n, betas = 4, 9, 6, [0.9, 1.4, 2.0]
    for k, r in enumerate(reals):
        J = oracle.ea_couplings(3, L, r, seed)
        s = np.stack([np.stack([oracle.ising_init(3, L, seed, oracle.lattice_id(a, r >> 5, t), bit=r & 31)
                                for t in range(3)]) for a in range(2)]).copy()
        E, Q, acc, _ = oracle.pt_run(3, L, s, betas, seed, r, r >> 5, 0, n, 1, J=J)
        ref = np.concatenate([E.ravel(), Q.ravel(), s.ravel().astype(np.int64)])
        assert np.array_equal(got[k], ref), r


def _slab_rank_main(rank, world, port, L, n, out_path):
    import torch
    import torch.distributed as dist
    import oracle
    from paper_1101_1427_gb300.slab import exchange_ghosts, split_rows
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    beta, seed = 0.44, 17
    lid = oracle.lattice_id(0, 0, 0)
    y0, rows = split_rows(L, world, rank)
    full0 = oracle.ising_init(2, L, seed, lid).reshape(L, L)
    slab = torch.zeros(rows + 2, L, dtype=torch.int8)
    slab[1:rows + 1] = torch.from_numpy(full0[y0:y0 + rows].copy())
    view = slab.numpy()  # shares memory with the tensor the exchange fills
    for sweep in range(n):
        for colour in (0, 1):
            exchange_ghosts(slab, rank, world)
            oracle.slab_phase(L, y0, rows, view, beta, seed, lid, sweep, colour)
    exchange_ghosts(slab, rank, world)
    # partial energy (bonds right and below of own sites) and magnetisation, then one all-reduce
    own, below = view[1:rows + 1].astype(np.int64), view[2:rows + 2].astype(np.int64)
    part = torch.tensor([-(own * np.roll(own, -1, axis=1)).sum() - (own * below).sum(), own.sum()],
                        dtype=torch.int64)
    dist.all_reduce(part)
    rows_all = [None] * world
    dist.all_gather_object(rows_all, view[1:rows + 1].copy())
    if rank == 0:
        np.savez(out_path, lattice=np.concatenate(rows_all), EM=part.numpy())
    dist.barrier()
    dist.destroy_process_group()


@pytest.mark.parametrize("world,L", [(2, 32), (3, 40)])
def test_slab_decomposition_over_gloo_ranks_equals_unsplit(world, L, tmp_path):
    """Ranks own bands of rows of one lattice and exchange one ghost row per
    neighbour before each colour phase (send/recv over gloo); the gathered
    lattice and the all-reduced E, M equal the unsplit oracle."""
    import torch.multiprocessing as mp
    import oracle
    n = 5
    out = tmp_path / "slab.npz"
    mp.start_processes(_slab_rank_main, args=(world, _free_port(), L, n, str(out)), nprocs=world,
                       join=True, start_method="spawn")
    res = np.load(out)
    lid = oracle.lattice_id(0, 0, 0)
    s = oracle.ising_init(2, L, 17, lid)
    for sweep in range(n):
        oracle.ising_sweep(2, L, s, 0.44, 17, lid, sweep)
    assert np.array_equal(res["lattice"].ravel(), s)
    assert res["EM"][0] == oracle.ising_energy(2, L, s)
    assert res["EM"][1] == oracle.ising_magnetisation(2, L, s)
