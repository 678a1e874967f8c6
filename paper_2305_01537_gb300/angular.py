"""Angular decomposition across ranks: the filter of a state whose shells are split in (theta, phi)
blocks over several processes (one per GPU).

The paper (Sec. II, "Filtering parallelization") runs the filter inside a domain decomposition in
(r, theta, phi): the processes of one radial range split each shell into angular blocks, and before
each pass the blocks are redistributed within the angular group so that every process holds whole
circles (theta pass) or whole rings (phi pass), then scattered back. Here one GPU filters whole
shells in one staging of both passes, so the analogue is a single exchange each way: an all-to-all
within the group gives every rank all angular blocks of a contiguous slab of radii (whole shells),
the rank filters its slab with its own plan, and a second all-to-all returns every rank's angular
block of every radius. The collective is the exchange step itself; the filter stays per shell.

Layouts (row-major, phi fastest): the caller's block is x[v][i][j][k] for all nvars fields and Nr
radii, rows j of the rank's theta range and columns k of its phi range; ranks are numbered
q = a * Pphi + b for theta block a and phi block b. Ranges split as evenly as possible (sizes differ
by at most one), so every rank may hold a different number of rows, columns and radii.
"""
from typing import Callable, List, Tuple

import torch
import torch.distributed as dist


def split_range(n: int, parts: int, index: int) -> Tuple[int, int]:
    """[start, stop) of part `index` of `parts` nearly equal parts of range(n)."""
    base, extra = divmod(n, parts)
    start = index * base + min(index, extra)
    return start, start + base + (1 if index < extra else 0)


class AngularFilter:
    """Filters a (theta, phi)-decomposed state by redistributing it to whole-shell radial slabs.

    filter_slab(slab_start, slab_stop, x) must return the filter of x, the whole shells of radii
    [slab_start, slab_stop) of every field, shape [nvars][ns][Ntheta][Nphi] (for instance a Plan
    built for those radii, applied on this rank's GPU). `group` is the angular group (default: the
    whole job); its size must be Ptheta * Pphi.
    """

    def __init__(self, Nr: int, Ntheta: int, Nphi: int, nvars: int, Ptheta: int, Pphi: int,
                 filter_slab: Callable[[int, int, torch.Tensor], torch.Tensor], group=None):
        self.Nr, self.Nth, self.Nph, self.nvars = Nr, Ntheta, Nphi, nvars
        self.Pth, self.Pph = Ptheta, Pphi
        self.group = group
        self.size = dist.get_world_size(group)
        self.rank = dist.get_rank(group)
        if self.size != Ptheta * Pphi:
            raise ValueError(f"angular group of {self.size} ranks, expected {Ptheta} x {Pphi}")
        if Ptheta > Ntheta or Pphi > Nphi or self.size > Nr:
            raise ValueError("more blocks than rows, columns or radii")
        self.filter_slab = filter_slab

    def block(self, q: int) -> Tuple[Tuple[int, int], Tuple[int, int]]:
        """Theta rows and phi columns ([start, stop) each) held by rank q."""
        a, b = divmod(q, self.Pph)
        return split_range(self.Nth, self.Pth, a), split_range(self.Nph, self.Pph, b)

    def slab(self, q: int) -> Tuple[int, int]:
        """Radii [start, stop) that rank q filters."""
        return split_range(self.Nr, self.size, q)

    def local_shape(self) -> Tuple[int, int, int, int]:
        (j0, j1), (k0, k1) = self.block(self.rank)
        return (self.nvars, self.Nr, j1 - j0, k1 - k0)

    def _exchange(self, send_parts: List[torch.Tensor], recv_sizes: List[int], like: torch.Tensor) -> List[torch.Tensor]:
        send = torch.cat([p.reshape(-1) for p in send_parts])
        recv = torch.empty(sum(recv_sizes), dtype=like.dtype, device=like.device)
        dist.all_to_all_single(recv, send, output_split_sizes=recv_sizes,
                               input_split_sizes=[p.numel() for p in send_parts], group=self.group)
        return list(torch.split(recv, recv_sizes))

    def apply(self, x_local: torch.Tensor) -> torch.Tensor:
        """The filter of the distributed state; x_local is this rank's block (local_shape())."""
        if tuple(x_local.shape) != self.local_shape():
            raise ValueError(f"block of shape {tuple(x_local.shape)}, expected {self.local_shape()}")
        x_local = x_local.contiguous()
        P, nv = self.size, self.nvars
        me_i0, me_i1 = self.slab(self.rank)
        ns = me_i1 - me_i0
        # 1. to whole shells: rank q receives every rank's block of q's radii
        send = [x_local[:, slice(*self.slab(q))] for q in range(P)]
        sizes = []
        for p in range(P):
            (j0, j1), (k0, k1) = self.block(p)
            sizes.append(nv * ns * (j1 - j0) * (k1 - k0))
        parts = self._exchange(send, sizes, x_local)
        full = torch.empty((nv, ns, self.Nth, self.Nph), dtype=x_local.dtype, device=x_local.device)
        for p in range(P):
            (j0, j1), (k0, k1) = self.block(p)
            full[:, :, j0:j1, k0:k1] = parts[p].view(nv, ns, j1 - j0, k1 - k0)
        # 2. the filter of this rank's slab of whole shells
        y = self.filter_slab(me_i0, me_i1, full)
        # 3. back to angular blocks: rank p receives its block of every slab
        send = []
        for p in range(P):
            (j0, j1), (k0, k1) = self.block(p)
            send.append(y[:, :, j0:j1, k0:k1].contiguous())
        (j0, j1), (k0, k1) = self.block(self.rank)
        sizes = []
        for q in range(P):
            i0, i1 = self.slab(q)
            sizes.append(nv * (i1 - i0) * (j1 - j0) * (k1 - k0))
        parts = self._exchange(send, sizes, x_local)
        out = torch.empty_like(x_local)
        for q in range(P):
            i0, i1 = self.slab(q)
            out[:, i0:i1] = parts[q].view(nv, i1 - i0, j1 - j0, k1 - k0)
        return out


def plan_slab_filter(grid, precision: int = 0):
    """A filter_slab for AngularFilter that runs this rank's CUDA plan: one Plan per slab of radii
    (the grid's parity, kinds, cutoffs and radii r[start:stop]), built on first use on the current
    device. The slab arrives as host or device FP64 data; the result is returned on the same device."""
    from .binding import Plan
    plans = {}

    def run(i0: int, i1: int, x: torch.Tensor) -> torch.Tensor:
        key = (i0, i1)
        if key not in plans:
            plans[key] = Plan(i1 - i0, grid.Ntheta, grid.Nphi, grid.parity, grid.kind, grid.L,
                              grid.r[i0:i1], grid.dr_min, grid.floor, precision, getattr(grid, "eps", 1e-12))
        dev = x.device
        y = plans[key].apply(x.to(device=f"cuda:{plans[key].device}", dtype=torch.float64).contiguous())
        return y.to(dev)

    return run
