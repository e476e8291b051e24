"""Slab decomposition of one 2D int8 ferromagnet over several ranks (GPUs):
rank k owns a band of rows and keeps it with one ghost row above and below,
[rows + 2][L] int8.  Before every colour phase each rank sends its first own
row to the rank above and its last own row to the rank below, and receives
its ghosts from them (periodic in y); the phase itself is spin_slab_phase,
whose random words are keyed by global site index, so the split chain is the
unsplit one.  Energies and magnetisations are per-slab partial sums
(spin_slab_measure) to be all-reduced."""
import torch

from . import _binding as B


def split_rows(L, world, rank):
    """Rows [y0, y0 + rows) of rank `rank` (heights differ by at most one)."""
    y0 = round(rank * L / world)
    return y0, round((rank + 1) * L / world) - y0


def exchange_ghosts(slab, rank, world, group=None):
    """Fill the two ghost rows of `slab` from the neighbouring ranks.  Sends
    go up then down and receives come from below then above, so that with
    two ranks (one peer on both sides) the messages pair in order."""
    import torch.distributed as dist
    if world == 1:
        slab[0].copy_(slab[-2])
        slab[-1].copy_(slab[1])
        return
    up, down = (rank - 1) % world, (rank + 1) % world
    first, last = slab[1].contiguous(), slab[-2].contiguous()
    top, bottom = torch.empty_like(first), torch.empty_like(first)
    ops = [dist.P2POp(dist.isend, first, up, group, tag=0),
           dist.P2POp(dist.isend, last, down, group, tag=1),
           dist.P2POp(dist.irecv, bottom, down, group, tag=0),
           dist.P2POp(dist.irecv, top, up, group, tag=1)]
    for req in dist.batch_isend_irecv(ops):
        req.wait()
    slab[0].copy_(top)
    slab[-1].copy_(bottom)


def exchange_ghosts_local(slabs):
    """The same exchange among slabs held by one process (one GPU emulating
    several ranks, or a test)."""
    P = len(slabs)
    tops = [slabs[k - 1][-2].clone() for k in range(P)]
    bottoms = [slabs[(k + 1) % P][1].clone() for k in range(P)]
    for sl, t, b in zip(slabs, tops, bottoms):
        sl[0].copy_(t)
        sl[-1].copy_(b)


def phase(slab, L, y0, rows, beta, seed, lattice_id, sweep, colour, stream=None):
    stream = stream or torch.cuda.current_stream()
    B.spin_slab_phase(slab, L, y0, rows, beta, seed, lattice_id, sweep, colour, stream.cuda_stream)


def measure(slab, L, rows, E, M, stream=None):
    stream = stream or torch.cuda.current_stream()
    B.spin_slab_measure(slab, L, rows, E, M, stream.cuda_stream)
