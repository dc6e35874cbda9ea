"""Row-slab domain decomposition of one cavity (argument marshalling and message routing).

The fused step pulls every population from the previous state of a
neighbouring node, so a cavity split into horizontal slabs of rows needs, per
time step and per cut, only the populations that cross the cut: per node
f2, f5, f6, g2 upward and f4, f7, f8, g4 downward (3 D2Q9 + 1 D2Q5 each way).
Each slab is a library context with a ghost row beyond each cut
(``lbm_init_slab``); after every step the outgoing populations are packed
(``lbm_halo_pack``), moved to the neighbour, and unpacked into its ghost row
(``lbm_halo_unpack``).  The wall Nusselt number and the convergence residual
become sums over each slab's interior rows, added up across slabs.

Two drivers:

* :class:`SlabRun` -- several slabs in one process on one device and one
  stream; the messages are device buffers read in place.
* :class:`DistributedSlab` -- one slab per rank of a ``torch.distributed``
  group; the messages go by point-to-point send/recv (NCCL between GPUs) and
  the sums by an all-reduce.

All arithmetic runs in the library; this module only routes buffers.
"""
from __future__ import annotations

import math

import numpy as np

from . import lbm


def partition(ny: int, parts: int):
    """Row ranges [(y0, y1), ...] of `parts` slabs as equal as possible."""
    if parts < 1 or parts > ny:
        raise ValueError("need 1 <= parts <= ny")
    base, extra = divmod(ny, parts)
    out, y = [], 0
    for p in range(parts):
        h = base + (1 if p < extra else 0)
        out.append((y, y + h))
        y += h
    return out


def combine_residual(sums):
    """r = max over (u_x, u_y, T) of sqrt(sum (phi - phi_prev)^2 / sum phi^2)
    from the seven added-up sums of lbm_residual_sums, and the non-finite count."""
    s = np.asarray(sums, dtype=np.float64)
    r = 0.0
    for c in range(3):
        num, den = s[2 * c], s[2 * c + 1]
        v = math.sqrt(num / den) if den > 0 else (math.inf if num > 0 else 0.0)
        r = max(r, v)
    return r, float(s[6])


class _LibSlab:
    """The library calls of one slab context (the operations the drivers route)."""

    def __init__(self, nx, ny, y0, y1, params, **opts):
        self.ctx = lbm.init_slab(nx, ny, y0, y1, params["n"], params["Da"], params["Ra"], params["Pr"],
                                 params.get("porosity", 0.6), **opts)
        self.y0, self.row_lo, self.row_hi, self.ny_local = lbm.slab_rows(self.ctx)
        self.nx = nx
        self.halo_bytes = lbm.halo_bytes(self.ctx)

    def close(self):
        if self.ctx:
            lbm.destroy(self.ctx)
            self.ctx = None

    def step(self, k):
        lbm.step(self.ctx, k)

    def pack(self, d_lo, d_hi):
        lbm.halo_pack(self.ctx, d_lo, d_hi)

    def unpack(self, d_lo, d_hi):
        lbm.halo_unpack(self.ctx, d_lo, d_hi)

    def nusselt_sums(self):
        return lbm.nusselt_sums(self.ctx)

    def residual_sums(self):
        return lbm.residual_sums(self.ctx)

    def synchronize(self):
        lbm.synchronize(self.ctx)


class SlabRun:
    """An nx x ny cavity as `parts` row slabs on one device and one stream.

    ``stream`` (a torch.cuda.Stream or a cudaStream_t) is shared by every
    slab so that steps, packs and unpacks run in the order they are queued;
    the message buffers are torch device tensors.  Results equal the
    undivided cavity's (bit for bit with FP64 and FP32 storage).
    """

    def __init__(self, nx, ny, parts, n, Da, Ra, Pr, porosity=0.6, stream=None, device=0, **opts):
        import torch
        self.nx, self.ny = nx, ny
        self.bounds = partition(ny, parts)
        if stream is None:
            stream = torch.cuda.Stream(device=device)
        self._stream = stream
        params = dict(n=n, Da=Da, Ra=Ra, Pr=Pr, porosity=porosity)
        self.slabs = [_LibSlab(nx, ny, y0, y1, params, cuda_stream=stream, device=device, **opts)
                      for y0, y1 in self.bounds]
        hb = self.slabs[0].halo_bytes
        # up[i]: message from slab i to slab i + 1; down[i]: from slab i + 1 to slab i
        self.up = [torch.empty(hb, dtype=torch.uint8, device=f"cuda:{device}") for _ in self.bounds[1:]]
        self.down = [torch.empty(hb, dtype=torch.uint8, device=f"cuda:{device}") for _ in self.bounds[1:]]
        self.exchange()

    def close(self):
        for s in self.slabs:
            s.close()

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def exchange(self):
        """Refresh every ghost row from the neighbours' current states."""
        last = len(self.slabs) - 1
        for i, s in enumerate(self.slabs):
            s.pack(self.down[i - 1].data_ptr() if i > 0 else None, self.up[i].data_ptr() if i < last else None)
        for i, s in enumerate(self.slabs):
            s.unpack(self.up[i - 1].data_ptr() if i > 0 else None, self.down[i].data_ptr() if i < last else None)

    def step(self, k: int = 1):
        for _ in range(int(k)):
            for s in self.slabs:
                s.step(1)
            self.exchange()

    def nusselt(self):
        """(hot-wall, cold-wall) average Nu of the whole cavity."""
        h = c = 0.0
        for s in self.slabs:
            a, b = s.nusselt_sums()
            h += a
            c += b
        return h / self.ny, c / self.ny

    def residual(self):
        tot = np.zeros(7)
        for s in self.slabs:
            tot += s.residual_sums()
        return combine_residual(tot)[0]

    def interior(self, arrays_of_slab):
        """Stack the interior rows of per-slab arrays [..., ny_local, nx] into [..., ny, nx]."""
        return np.concatenate([a[..., s.row_lo:s.row_hi, :] for s, a in zip(self.slabs, arrays_of_slab)],
                              axis=-2)

    def get_state_f64(self):
        parts = [lbm.get_state_f64(s.ctx, self.nx, s.ny_local) for s in self.slabs]
        return tuple(self.interior([p[j] for p in parts]) for j in range(3))

    def set_state_f64(self, f, g, tau):
        """Set the whole cavity's state (each slab takes its rows and ghosts)."""
        for s, (y0, y1) in zip(self.slabs, self.bounds):
            lo, hi = y0 - s.row_lo, y0 - s.row_lo + s.ny_local
            lbm.set_state_f64(s.ctx, f[:, lo:hi], g[:, lo:hi], tau[lo:hi])
        self.exchange()


class DistributedSlab:
    """This rank's slab of an nx x ny cavity split over the ranks of a
    ``torch.distributed`` group (rank r holds partition(ny, world)[r]).

    Every step: the library steps the slab, packs the two outgoing messages,
    they go to the ranks above and below by send/recv, and the received ones
    are unpacked into the ghost rows.  With NCCL the message tensors live on
    this rank's GPU and the library runs on torch's current stream, so the
    packs, the transfers and the unpacks are stream-ordered.  ``ops`` and
    ``make_buffer`` replace the library slab and the tensor allocation (the
    routing is independent of where the slab's arithmetic runs).
    """

    def __init__(self, nx, ny, n, Da, Ra, Pr, porosity=0.6, group=None, ops=None, make_buffer=None, **opts):
        import torch
        import torch.distributed as dist
        self.dist, self.torch, self.group = dist, torch, group
        self.rank = dist.get_rank(group)
        self.world = dist.get_world_size(group)
        self.nx, self.ny = nx, ny
        self.y0, self.y1 = partition(ny, self.world)[self.rank]
        if ops is None:
            dev = torch.cuda.current_device()
            ops = _LibSlab(nx, ny, self.y0, self.y1, dict(n=n, Da=Da, Ra=Ra, Pr=Pr, porosity=porosity),
                           cuda_stream=torch.cuda.current_stream(), device=dev, **opts)
            make_buffer = make_buffer or (lambda nb: torch.empty(nb, dtype=torch.uint8, device=f"cuda:{dev}"))
        self.ops = ops
        make_buffer = make_buffer or (lambda nb: torch.empty(nb, dtype=torch.uint8))
        hb = ops.halo_bytes
        self.has_lo, self.has_hi = self.rank > 0, self.rank < self.world - 1
        self.send_lo = make_buffer(hb) if self.has_lo else None
        self.recv_lo = make_buffer(hb) if self.has_lo else None
        self.send_hi = make_buffer(hb) if self.has_hi else None
        self.recv_hi = make_buffer(hb) if self.has_hi else None
        self.exchange()

    def _peer(self, r):
        return r if self.group is None else self.dist.get_global_rank(self.group, r)

    @staticmethod
    def _ptr(t):
        return None if t is None else t.data_ptr()

    def exchange(self):
        """Send this slab's cut populations to the neighbours and fill the
        ghost rows with theirs (nothing to do for a single slab)."""
        if not (self.has_lo or self.has_hi):
            return
        self.ops.pack(self._ptr(self.send_lo), self._ptr(self.send_hi))
        ops = []
        P2P = self.dist.P2POp
        if self.has_lo:
            ops += [P2P(self.dist.isend, self.send_lo, self._peer(self.rank - 1), self.group),
                    P2P(self.dist.irecv, self.recv_lo, self._peer(self.rank - 1), self.group)]
        if self.has_hi:
            ops += [P2P(self.dist.isend, self.send_hi, self._peer(self.rank + 1), self.group),
                    P2P(self.dist.irecv, self.recv_hi, self._peer(self.rank + 1), self.group)]
        if ops:
            for req in self.dist.batch_isend_irecv(ops):
                req.wait()
        self.ops.unpack(self._ptr(self.recv_lo), self._ptr(self.recv_hi))

    def step(self, k: int = 1):
        for _ in range(int(k)):
            self.ops.step(1)
            self.exchange()

    def _all_sum(self, values):
        t = self.torch.tensor(np.asarray(values, dtype=np.float64))
        if self.dist.get_backend(self.group) == "nccl":
            t = t.cuda()
        self.dist.all_reduce(t, group=self.group)
        return t.cpu().numpy()

    def nusselt(self):
        """(hot-wall, cold-wall) average Nu of the whole cavity (an all-reduce)."""
        h, c = self._all_sum(self.ops.nusselt_sums())
        return float(h) / self.ny, float(c) / self.ny

    def residual(self):
        """Convergence residual of the whole cavity (an all-reduce of seven sums)."""
        return combine_residual(self._all_sum(self.ops.residual_sums()))[0]
