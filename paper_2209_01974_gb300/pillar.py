"""Pillar layout of the FD search block over ranks (Sec. 3.4, 3.5).

In the paper's pillar layout every process holds the whole matrix and a
contiguous share of the N_s search vectors, in bundles of n_b columns; the
polynomial filter then needs no communication at all, and the only exchange of
an outer iteration is the redistribution of the filtered vectors before the
orthogonalisation and the Rayleigh-Ritz step.  Here one rank runs per GPU:

* ``bundle_ranges`` splits the N_s / n_b bundles into contiguous, balanced
  column ranges, one per rank;
* ``filter_own`` applies the rank's filter (``fd_filter`` on its GPU, or any
  callable with the same effect) to its own bundles;
* ``gather_columns`` all-gathers the filtered column ranges so that every rank
  holds the whole block (``torch.distributed``: NCCL between GPUs, gloo on
  CPU);
* ``pillar_step`` is one outer iteration's filter + exchange, after which every
  rank repeats the same orthonormalisation and Rayleigh-Ritz step on identical
  data, so the ranks stay in lockstep without a second exchange.

This module holds bookkeeping and communication only; the arithmetic is the
caller's filter and dense steps.
"""


def bundle_ranges(ns, nb, world):
    """Column range (c0, c1) of each rank: the ns / nb bundles split into world
    contiguous groups whose sizes differ by at most one bundle (a rank without a
    bundle gets an empty range)."""
    if ns % nb:
        raise ValueError("ns must be a multiple of nb")
    if world < 1:
        raise ValueError("world must be >= 1")
    nbund = ns // nb
    base, extra = divmod(nbund, world)
    out, b0 = [], 0
    for r in range(world):
        k = base + (1 if r < extra else 0)
        out.append((b0 * nb, (b0 + k) * nb))
        b0 += k
    return out


def filter_own(V, own, nb, filter_fn):
    """Apply filter_fn(columns) in place to each nb-wide bundle of the rank's
    column range own = (c0, c1) of V (D x N_s)."""
    c0, c1 = own
    for j in range(c0, c1, nb):
        filter_fn(V[:, j:j + nb])


def gather_columns(V, ranges, rank, group=None):
    """All-gather: afterwards every rank's V holds every rank's column range
    (V is D x N_s, each rank having written its own range).  Ranges may be
    uneven; they are padded to the widest for the collective."""
    import torch
    import torch.distributed as dist
    width = max(c1 - c0 for c0, c1 in ranges)
    if width == 0:
        return V
    D = V.shape[0]
    c0, c1 = ranges[rank]
    mine = torch.zeros((D, width), dtype=V.dtype, device=V.device)
    mine[:, :c1 - c0] = V[:, c0:c1]
    parts = [torch.empty_like(mine) for _ in ranges]
    dist.all_gather(parts, mine.contiguous(), group=group)
    for (a, b), part in zip(ranges, parts):
        V[:, a:b] = part[:, :b - a]
    return V


def pillar_step(V, nb, filter_fn, rank, world, group=None):
    """One outer iteration's distributed part: the rank filters its own bundles
    (no communication), then the ranks exchange their columns.  Returns the
    column ranges used."""
    ranges = bundle_ranges(V.shape[1], nb, world)
    filter_own(V, ranges[rank], nb, filter_fn)
    if world > 1:
        gather_columns(V, ranges, rank, group)
    return ranges
