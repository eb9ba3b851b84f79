"""Splitting one DOS over several processes (one GPU each) by k-slabs.

The Brillouin-zone sum of Eqs. (8)-(9) runs over cubes, so the cube planes
z in [0, n3) can be cut into contiguous slabs, each integrated by its own
plan (``tetra_desc_t.z_begin/z_end``) on its own GPU. Every rank computes H(k)
and the eigen-data for its slab plus one halo plane itself, so the only
exchange is the final sum of the [n_orb][n_omega] slab results, done here in
rank order so that every rank gets the same bits.
"""
from __future__ import annotations


def slab_ranges(n3: int, world: int) -> list[tuple[int, int]]:
    """Contiguous cube-plane ranges [z0, z1) for `world` ranks, sizes differing
    by at most one; ranks beyond n3 get empty ranges (z0 == z1)."""
    if n3 < 1 or world < 1:
        raise ValueError("n3 and world must be positive")
    base, extra = divmod(n3, world)
    out, z = [], 0
    for r in range(world):
        size = base + (1 if r < extra else 0)
        out.append((z, z + size))
        z += size
    return out


def combine_slabs(torch, parts):
    """Sum of per-slab DOS arrays in the given (rank) order, in float64, cast
    to float32."""
    acc = torch.zeros(parts[0].shape, dtype=torch.float64, device=parts[0].device)
    for p in parts:
        acc += p.to(torch.float64)
    return acc.to(torch.float32)


def gather_slabs(local_dos, group=None):
    """All ranks' slab DOS summed in rank order (an all-gather, then an ordered
    local sum: deterministic and identical on every rank). A rank with an empty
    slab passes zeros."""
    import torch
    import torch.distributed as dist
    world = dist.get_world_size(group)
    parts = [torch.empty_like(local_dos) for _ in range(world)]
    dist.all_gather(parts, local_dos.contiguous(), group=group)
    return combine_slabs(torch, parts)


def slab_dos(T, rank: int, world: int, n, n_bands, n_orb, n_omega, params, R, omega,
             mode: str = "point", weight_dtype: str = "f32", group=None):
    """This rank's slab of the DOS of a tight-binding model, summed over all
    ranks (every rank returns the full [n_orb][n_omega] result). The
    eigen-data of the slab are computed on this rank's GPU."""
    import torch
    z0, z1 = slab_ranges(n[2], world)[rank]
    if z1 > z0:
        plan = T.Plan(*n, n_bands, n_orb, n_omega, mode=mode, weight_dtype=weight_dtype,
                      z_range=(z0, z1))
        eps, w = plan.eig(params, R)
        local = plan.dos(eps, w, omega)
    else:
        local = torch.zeros((n_orb, n_omega), dtype=torch.float32, device=omega.device)
    return gather_slabs(local, group)
