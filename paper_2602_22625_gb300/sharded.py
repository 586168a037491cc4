"""Shared-parameter sharding of one canvas across ranks (one process per GPU).

The forward composites tiles independently (Sec. 3.1.1, "Parallelization") and the
loss is a sum over pixels, so one canvas splits into horizontal bands of whole tile
rows, one band per rank, with every rank holding all primitives and the same
parameters.  Each rank bins the whole canvas, then composites and differentiates
only its band (dbmp_batch_set_rows); the fused MSE keeps its normalisation over the
whole canvas, so the bands' losses and parameter gradients (Eq. 6 summed over the
band's pixels) add up to the whole canvas' exactly up to summation order.  The one
exchange of a step is a sum all-reduce of the N x 8 gradient; every rank then takes
the same Adam step.

This module holds the partition and the exchange only: every arithmetic step of a
band runs in libdbmp's kernels, the sum in torch.distributed (NCCL on GPUs, gloo on
CPU).
"""
from __future__ import annotations


def band_rows(H: int, world: int, rank: int, tile: int = 32) -> tuple[int, int]:
    """Rows [y0, y1) of rank's band: the canvas' tile rows split as evenly as
    possible, earlier ranks taking one more when they do not divide.  Both ends are
    multiples of the tile size (y1 may pass H on the last ragged tile row)."""
    if world < 1 or not 0 <= rank < world:
        raise ValueError(f"rank {rank} outside 0..{world - 1}")
    nty = -(-H // tile)
    per, extra = divmod(nty, world)
    t0 = rank * per + min(rank, extra)
    t1 = t0 + per + (1 if rank < extra else 0)
    return t0 * tile, t1 * tile


def select_band(ws, H: int, world: int, rank: int, tile: int):
    """Restricts the workspace's plan to rank's band; returns its rows."""
    from . import dbmp as D
    y0, y1 = band_rows(H, world, rank, tile)
    if world == 1:
        D.dbmp_batch_set_rows(ws, 0, 0)
    elif y0 < y1:
        D.dbmp_batch_set_rows(ws, y0, y1)
    else:   # more ranks than tile rows: an empty band, one tile row past the canvas
        end = -(-H // tile) * tile
        D.dbmp_batch_set_rows(ws, end, end + tile)
    return y0, y1


def sum_gradient_(grad, world: int, group=None):
    """grad <- the sum of grad over the ranks of the process group (in place)."""
    if world > 1:
        import torch.distributed as dist
        dist.all_reduce(grad, op=dist.ReduceOp.SUM, group=group)
    return grad
