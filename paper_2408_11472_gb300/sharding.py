"""Sharding one realization's scatterers over ranks, then one sum-reduce of the spectra.

This is the data-parallel split of Section II.B (Fig. 2): the devices divide the
scatterer tiles, each computes a partial result, and the partials are added.  Because the
summation outputs accumulate (``+=``), a rank's partial spectra over its tile range are
plain additive terms: one all-reduce (SUM) of the [S, N_g, N_d] spectra (4.3 MB for 65
spectra of 128 x 64) completes them before the post-processing, which is cheap enough to
run replicated.

Shard boundaries are multiples of the library's scatterer block (``block_scatterers()``,
the set of consecutive scatterers that shares one FP64 reference point), so every
scatterer sees the same reference point and takes the same FP32 index decisions as in an
unsharded run.  The per-rank fixed-point sums are exact; only the final floating-point
all-reduce can differ in the last bits from a single-device run.
"""
from __future__ import annotations

from typing import Callable, Tuple

from . import _lib


def block_scatterers() -> int:
    """Scatterers per block sharing one FP64 reference point (CTA chunk of the kernels)."""
    return int(_lib.lib.rsim_block_scatterers())


def shard_range(n: int, world: int, rank: int, align: int | None = None) -> Tuple[int, int]:
    """[start, stop) of rank's share of n scatterers: contiguous, disjoint, covering [0, n),
    boundaries at multiples of ``align`` (default: block_scatterers()), as even as possible."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError("rank %d outside world of size %d" % (rank, world))
    a = block_scatterers() if align is None else int(align)
    blocks = (n + a - 1) // a
    base, extra = divmod(blocks, world)
    b0 = rank * base + min(rank, extra)
    b1 = b0 + base + (1 if rank < extra else 0)
    return min(n, b0 * a), min(n, b1 * a)


def sharded_spectra(partial_fn: Callable[[int, int], "object"], n: int, world: int, rank: int,
                    group=None, align: int | None = None):
    """Spectra of all n scatterers: ``partial_fn(start, stop)`` computes this rank's partial
    spectra (a torch tensor) over its shard; one all-reduce (SUM) completes them on every rank."""
    import torch.distributed as dist

    start, stop = shard_range(n, world, rank, align)
    T = partial_fn(start, stop)
    if world > 1:
        dist.all_reduce(T, op=dist.ReduceOp.SUM, group=group)
    return T
