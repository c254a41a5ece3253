"""One text split across ranks (GPUs): contiguous slices, one exchange step.

Sect. 3.2: the chunks of the parallel parser depend on one another only
through the join (Eq. joiner).  A text split into contiguous slices, one per
rank, is parsed in three steps (the library's sharded-parse calls):

1. every rank computes its slice's maps (``Regex.shard_map``): the forward
   state at the slice's end for every forward state at its start, and the
   backward state at its start for every backward state at its end -- a few
   hundred bytes, independent of the slice's length;
2. the maps are all-gathered (``gather_maps``: the only collective, on the
   process group's backend) and every rank composes them in order on the host
   (``Regex.shard_entry``) into each slice's exact entry states and the
   text's verdict;
3. every rank parses its slice from its entry states (``Regex.parse_slice``):
   its columns are those of the whole text's SLPF.

Argument marshalling and the exchange only; every step of the parse runs in
the library's kernels.
"""
from __future__ import annotations

import numpy as np


def slice_bounds(n: int, parts: int, align: int = 64):
    """Slice starts and ends of an n-byte text in ``parts`` near-equal
    slices starting at multiples of ``align`` (the library wants 16-byte
    aligned text pointers); empty slices are dropped."""
    cuts = [0] + [min(n, (n * r // parts) // align * align) for r in range(1, parts)] + [n]
    return [(a, b) for a, b in zip(cuts[:-1], cuts[1:]) if b > a]


def gather_maps(local_map: np.ndarray, group=None) -> np.ndarray:
    """All-gather every rank's slice maps (the exchange step): a [ranks,
    entries] uint8 array in rank order.  Single process: the map alone."""
    import torch
    import torch.distributed as dist
    m = np.ascontiguousarray(local_map, dtype=np.uint8)
    if not (dist.is_available() and dist.is_initialized()):
        return m[None, :]
    world = dist.get_world_size(group)
    dev = torch.device("cuda", torch.cuda.current_device()) if dist.get_backend(group) == "nccl" else torch.device("cpu")
    t = torch.from_numpy(m).to(dev)
    out = [torch.empty_like(t) for _ in range(world)]
    dist.all_gather(out, t, group=group)
    return np.stack([o.cpu().numpy() for o in out])


def parse_sharded(rx, text_slice, prev: bool, nxt: bool, group=None, stream=None):
    """This rank's part of a sharded parse.  ``text_slice``: this rank's
    slice as a CUDA uint8 view whose byte before (prev) and after (nxt) are
    readable.  Returns (columns, status, accepted): the slice's len + 1
    columns of the whole text's SLPF, its status word (a tensor) and the
    text's verdict."""
    import torch.distributed as dist
    local = rx.shard_map(text_slice, prev, nxt, stream=stream)
    maps = gather_maps(local, group)
    rank = dist.get_rank(group) if (dist.is_available() and dist.is_initialized()) else 0
    entry, entry_bwd, accepted = rx.shard_entry(maps)
    cols, status, _ = rx.parse_slice(text_slice, int(entry[rank]), int(entry_bwd[rank]), stream=stream)
    return cols, status, accepted


def parse_in_slices(rx, text, parts: int):
    """The sharded parse of a whole CUDA text on this one device, slice after
    slice (the same three steps, the exchange being a stack): returns the
    stitched columns (a CUDA tensor of n + 1 columns), the slices' status
    words and the verdict."""
    import torch
    n = text.numel()
    bounds = slice_bounds(n, parts)
    maps = np.stack([rx.shard_map(text[a:b], a > 0, b < n) for a, b in bounds])
    entry, entry_bwd, accepted = rx.shard_entry(maps)
    cols, stats = [], []
    for r, (a, b) in enumerate(bounds):
        c, st, _ = rx.parse_slice(text[a:b], int(entry[r]), int(entry_bwd[r]))
        cols.append(c if r == len(bounds) - 1 else c[:-1])      # column b is slice r+1's column 0
        stats.append(st)
    return torch.cat(cols), torch.cat(stats), accepted
