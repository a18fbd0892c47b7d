"""Radial-shell sharding of one solve across ranks (one slab of shells per rank).

GenASiS II divides the mesh among processes into radial shells that each cover the full
solid angle (Sec. 2.1) and combines the moment sums across processes (Sec. 2.2).  Here
the combination is the one exchange the radial recurrences need: every slab's totals
T[2][K_L] (the sums of W^R A and of W^I A over its shells, from mp_slab_moments) go
through an exclusive prefix over the slabs in radial order -- 2 K_L doubles per rank --
and each slab finishes with mp_slab_potential(outer).  No other data crosses ranks.

    mesh = multipole.Mesh(r, theta, phi, L, G, precision, slab=slab_of(n_r, rank, world))
    mesh.set_density(rho_slab); mesh.set_phi_output(phi_slab)
    mesh.slab_moments(totals)
    outer = exchange_slab_totals(totals.view(2, -1))
    mesh.slab_potential(outer.reshape(-1))
"""
from __future__ import annotations


def slab_of(n_r: int, rank: int, world: int):
    """Shells [i0, i1) of rank `rank` when n_r shells are dealt to `world` ranks in radial
    order, the first n_r % world ranks taking one shell more."""
    if not 0 <= rank < world or n_r < world:
        raise ValueError(f"cannot give each of {world} ranks a shell of {n_r}")
    base, extra = divmod(n_r, world)
    i0 = rank * base + min(rank, extra)
    return i0, i0 + base + (1 if rank < extra else 0)


def outer_from_totals(all_totals, rank: int):
    """outer[2][K_L] of slab `rank` from every slab's totals all_totals[world][2][K_L] (radial
    order): the regular sums of the slabs below it, added outward, and the irregular sums of
    the slabs above it, added inward (the order the recurrences themselves run)."""
    import torch
    world = all_totals.shape[0]
    out = torch.zeros_like(all_totals[0])
    for r in range(rank):
        out[0] += all_totals[r, 0]
    for r in range(world - 1, rank, -1):
        out[1] += all_totals[r, 1]
    return out


def exchange_slab_totals(totals, group=None):
    """The exclusive prefix over ranks: every rank's totals [2][K_L] (float64, on the device
    of the process group's backend) are gathered, and this rank's outer sums returned."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    rank = dist.get_rank(group)
    gathered = [torch.empty_like(totals) for _ in range(world)]
    dist.all_gather(gathered, totals.contiguous(), group=group)
    return outer_from_totals(torch.stack(gathered), rank)
