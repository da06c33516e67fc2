"""Work split over the processes of a torch.distributed group, one GPU each.

* One scene split by slabs of block columns (the library's
  itm_scene_set_shard): every process fuses the whole depth frame into its
  part (no data moves for allocation and integration); the raycast runs per
  part and the one exchange step follows, an all-gather of the parts' vertex
  and normal maps, then itm_raycast_merge on every process (per pixel, the
  hit nearest to the camera).  The collective runs on the group's backend
  (NCCL between GPUs, gloo on CPU).
* Independent scenes or submaps (the batched form): dealt to the processes
  by estimated size, largest first to the least loaded (no collective).
"""

from __future__ import annotations

import torch
import torch.distributed as dist


def slab_owner(bx: int, parts: int, slab_blocks: int) -> int:
    """Part that owns block column bx: floor(bx / slab_blocks) mod parts."""
    return (int(bx) // int(slab_blocks)) % int(parts)


def deal_by_size(sizes, parts: int):
    """Indices of `sizes` dealt to `parts` processes: largest first, each to
    the process with the least estimated work so far (ties: the lower
    process, then the lower index).  Returns one index list per process."""
    order = sorted(range(len(sizes)), key=lambda i: (-float(sizes[i]), i))
    load = [0.0] * int(parts)
    out = [[] for _ in range(int(parts))]
    for i in order:
        p = min(range(int(parts)), key=lambda k: (load[k], k))
        out[p].append(i)
        load[p] += float(sizes[i])
    return out


def exchange(mine_v: torch.Tensor, mine_n: torch.Tensor, group=None, out=None):
    """The exchange step: every process's vertex and normal map to every
    process.  Returns (vertex_parts, normal_parts) of shape (parts, *map),
    part k's maps at index k (written into `out` when given)."""
    parts = dist.get_world_size(group)
    shape = (parts,) + tuple(mine_v.shape)
    if out is None or out[0].shape != shape:
        out = (torch.empty(shape, dtype=mine_v.dtype, device=mine_v.device),
               torch.empty(shape, dtype=mine_n.dtype, device=mine_n.device))
    vparts, nparts = out
    dist.all_gather(list(vparts.unbind(0)), mine_v.contiguous(), group=group)
    dist.all_gather(list(nparts.unbind(0)), mine_n.contiguous(), group=group)
    return vparts, nparts


class ShardedScene:
    """This process's part of a scene split over `group` (default: the whole
    world).  `params` are the scene parameters of the whole scene."""

    def __init__(self, params, slab_blocks=8, group=None):
        from . import Scene
        self.group = group
        self.parts = dist.get_world_size(group)
        self.index = dist.get_rank(group)
        self.slab_blocks = int(slab_blocks)
        self.scene = Scene(**params)
        self.scene.set_shard(self.parts, self.index, self.slab_blocks)
        self._mine = None
        self._gathered = None

    def close(self):
        self.scene.close()

    def process(self, depth, intr, T_wc, vertex, normal, stream=None):
        """Allocate and integrate this part from the whole frame, raycast it,
        exchange the parts' maps and merge them into vertex / normal (device
        float32 [H, W, 4]) on every process."""
        from . import itm_raycast_merge
        if self._mine is None or self._mine[0].shape != vertex.shape or self._mine[0].device != vertex.device:
            self._mine = (torch.empty_like(vertex), torch.empty_like(normal))
        mine_v, mine_n = self._mine
        self.scene.process(depth, intr, T_wc, mine_v, mine_n, stream)
        self._gathered = exchange(mine_v, mine_n, self.group, self._gathered)
        vparts, nparts = self._gathered
        itm_raycast_merge(vparts, nparts, self.parts, intr, T_wc, vertex, normal, stream)
