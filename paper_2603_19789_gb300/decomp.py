"""Sharding across ranks (host side, torch.distributed): replica timing and the domain
decomposition of one grid.

Replicas.  `bench.py --gpus N` runs N independent copies of the workload; each rank times
its own run and the job's time is the maximum over ranks (`max_over_ranks`).

Domain decomposition.  One grid of nx x ny cells is cut into px x py blocks; rank
r = iy * px + ix owns rows [y0, y1) and columns [x0, x1).  The SSLBM step reads the four
lattice neighbours (Sec. II.B, D2Q5), so K steps read cells up to Manhattan distance K.
Before each block of K steps a rank receives a halo of width K from its neighbours (two
phases, along x then along y over the x-extended rows, which also fills the corners),
advances its extended block by K steps, and keeps the interior: after K steps every
interior cell is exact, whatever happened at the halo's outer edge.

At the global boundary:
  - periodic: every side has a neighbour (the wrap; a rank can be its own neighbour);
  - no-flux: a side on the global boundary gets no halo, and the step function applies the
    scheme's own no-flux rule there, exactly as the single-domain run does.
So the decomposed run computes each cell with the same operands in the same order as the
single-domain run: the results are bitwise identical.  Any step function that advances a
(C, ny, nx) block by K steps under a boundary rule can be used: the GPU solver on each
rank's device, or the CPU reference in the tests.
"""
from __future__ import annotations

from dataclasses import dataclass

import numpy as np

BC_PERIODIC, BC_NOFLUX = 0, 1


def max_over_ranks(x: float, world: int, device=None) -> float:
    """Maximum of a per-rank scalar over all ranks (the job's time of a replica run)."""
    if world == 1:
        return float(x)
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def split(n: int, parts: int):
    """[start, stop) bounds of `parts` nearly equal pieces of range(n)."""
    if parts < 1 or parts > n:
        raise ValueError(f"cannot split {n} cells into {parts} parts")
    q, r = divmod(n, parts)
    out, s = [], 0
    for i in range(parts):
        e = s + q + (1 if i < r else 0)
        out.append((s, e))
        s = e
    return out


@dataclass
class Decomposition:
    nx: int
    ny: int
    px: int
    py: int
    rank: int
    bc: int = BC_PERIODIC

    def __post_init__(self):
        if not 0 <= self.rank < self.px * self.py:
            raise ValueError("rank outside the px x py layout")
        self.ix, self.iy = self.rank % self.px, self.rank // self.px
        self.x0, self.x1 = split(self.nx, self.px)[self.ix]
        self.y0, self.y1 = split(self.ny, self.py)[self.iy]

    def rank_of(self, ix: int, iy: int) -> int:
        return iy * self.px + ix

    def neighbour(self, axis: int, side: int):
        """Rank across side (-1 or +1) along axis (0 = x, 1 = y); None at a no-flux edge."""
        i, p = (self.ix, self.px) if axis == 0 else (self.iy, self.py)
        j = i + side
        if j < 0 or j >= p:
            if self.bc == BC_NOFLUX:
                return None
            j %= p
        return self.rank_of(j, self.iy) if axis == 0 else self.rank_of(self.ix, j)

    def halo(self, K: int):
        """Halo widths (left, right, down, up): K towards a neighbour, 0 at a no-flux edge."""
        return tuple(0 if self.neighbour(ax, sd) is None else K for ax, sd in ((0, -1), (0, 1), (1, -1), (1, 1)))

    def local(self, full: np.ndarray) -> np.ndarray:
        """This rank's block of a (C, ny, nx) array."""
        return np.ascontiguousarray(full[:, self.y0:self.y1, self.x0:self.x1])

    def extend(self, block: np.ndarray, K: int) -> np.ndarray:
        hl, hr, hd, hu = self.halo(K)
        c, h, w = block.shape
        if min(h, w) < K:
            raise ValueError(f"block {h}x{w} is narrower than the halo width {K}")
        ext = np.zeros((c, h + hd + hu, w + hl + hr), dtype=block.dtype)
        ext[:, hd:hd + h, hl:hl + w] = block
        return ext

    def interior(self, ext: np.ndarray, K: int) -> np.ndarray:
        hl, hr, hd, hu = self.halo(K)
        h, w = self.y1 - self.y0, self.x1 - self.x0
        return np.ascontiguousarray(ext[:, hd:hd + h, hl:hl + w])

    def exchange(self, ext: np.ndarray, K: int) -> None:
        """Fill the halo of an extended block from the neighbours' interiors (collective:
        every rank calls it with the same K)."""
        import torch
        import torch.distributed as dist
        hl, hr, hd, hu = self.halo(K)
        h, w = self.y1 - self.y0, self.x1 - self.x0
        rows = slice(hd, hd + h)
        # phase x: interior rows; phase y: full extended width (fills the corners)
        for axis in (0, 1):
            if axis == 0:
                lo_send = ext[:, rows, hl:hl + K]            # my first K columns -> left neighbour
                hi_send = ext[:, rows, hl + w - K:hl + w]    # my last K columns -> right neighbour
                lo_dst = (slice(None), rows, slice(0, hl))
                hi_dst = (slice(None), rows, slice(hl + w, hl + w + hr))
                nlo, nhi = self.neighbour(0, -1), self.neighbour(0, 1)
                have_lo, have_hi = hl > 0, hr > 0
            else:
                lo_send = ext[:, hd:hd + K, :]
                hi_send = ext[:, hd + h - K:hd + h, :]
                lo_dst = (slice(None), slice(0, hd), slice(None))
                hi_dst = (slice(None), slice(hd + h, hd + h + hu), slice(None))
                nlo, nhi = self.neighbour(1, -1), self.neighbour(1, 1)
                have_lo, have_hi = hd > 0, hu > 0
            recv_lo = np.empty_like(ext[lo_dst]) if have_lo else None
            recv_hi = np.empty_like(ext[hi_dst]) if have_hi else None
            reqs, bufs = [], []
            # my low strip fills my low neighbour's high halo and my high strip its low halo;
            # the tag names the receiving halo (2 axis + 0 low / + 1 high), so the two
            # messages between a pair of ranks that are neighbours on both sides never mix
            for nb, send, recv, have, send_tag, recv_tag in (
                    (nlo, lo_send, recv_lo, have_lo, 2 * axis + 1, 2 * axis),
                    (nhi, hi_send, recv_hi, have_hi, 2 * axis, 2 * axis + 1)):
                if not have or nb == self.rank:
                    continue
                ts = torch.from_numpy(np.ascontiguousarray(send))
                tr = torch.from_numpy(recv)
                bufs += [ts, tr]
                reqs.append(dist.isend(ts, nb, tag=send_tag))
                reqs.append(dist.irecv(tr, nb, tag=recv_tag))
            for r in reqs:
                r.wait()
            # a rank that is its own neighbour (periodic, one block along this axis) wraps
            if have_lo:
                ext[lo_dst] = hi_send if nlo == self.rank else recv_lo
            if have_hi:
                ext[hi_dst] = lo_send if nhi == self.rank else recv_hi

    def gather(self, block: np.ndarray, root: int = 0):
        """The full (C, ny, nx) array on root (None elsewhere)."""
        import torch
        import torch.distributed as dist
        world = self.px * self.py
        c = block.shape[0]
        if self.rank != root:
            dist.send(torch.from_numpy(np.ascontiguousarray(block)), root)
            return None
        full = np.empty((c, self.ny, self.nx), dtype=block.dtype)
        for r in range(world):
            d = Decomposition(self.nx, self.ny, self.px, self.py, r, self.bc)
            if r == root:
                part = block
            else:
                t = torch.from_numpy(np.empty((c, d.y1 - d.y0, d.x1 - d.x0), dtype=block.dtype))
                dist.recv(t, r)
                part = t.numpy()
            full[:, d.y0:d.y1, d.x0:d.x1] = part
        return full


def run_decomposed(dec: Decomposition, block: np.ndarray, step, nsteps: int, K: int) -> np.ndarray:
    """Advance this rank's block by nsteps (blocks of K steps, the last one shorter):
    exchange a halo of width K, call step(ext, k, bc) -> ext advanced by k steps, keep
    the interior."""
    done = 0
    while done < nsteps:
        k = min(K, nsteps - done)
        ext = dec.extend(block, K)
        dec.exchange(ext, K)
        ext = step(ext, k, dec.bc)
        block = dec.interior(ext, K)
        done += k
    return block
