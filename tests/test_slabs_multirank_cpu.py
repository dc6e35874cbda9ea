"""Row-slab decomposition on CPU: gloo ranks route the halo messages and add
up the sums of paper_2011_15073_gb300.slabs.DistributedSlab.

The slab arithmetic runs in the CUDA library; here a numpy stand-in plays the
slab so that the routing -- which populations go to which rank, into which
ghost row -- and the reductions are checked without a GPU.  The stand-in
streams every population one node along its lattice velocity per step (the
pull of the fused step, bounce-back at the walls, no collision) in the
planes f0..f8, g0..g4 of the library's state, packs and unpacks the four
populations per cut node that lbm.h documents, and reports per-row sums as
its Nusselt and residual sums.  A decomposed run must equal the undivided one
on the interior rows; a wrong peer, a swapped side or a wrong ghost row
breaks that within a few steps.
"""
import os
import socket
import sys

import numpy as np
import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
torch = pytest.importorskip("torch")

E = [(0, 0), (1, 0), (0, 1), (-1, 0), (0, -1), (1, 1), (-1, 1), (-1, -1), (1, -1)]
OPP = [0, 3, 4, 1, 2, 7, 8, 5, 6]
VEL = E + E[:5]                    # planes f0..f8, g0..g4
OPPV = OPP + [0, 3, 4, 1, 2]
UP, DOWN = [2, 5, 6, 11], [4, 7, 8, 13]


class NumpySlab:
    """Stand-in for one slab context: state[14][ny_local][nx], ghost rows
    beyond the cuts, halo messages as bytes of [4][nx] float64."""

    def __init__(self, nx, ny, y0, y1, state_global):
        self.nx, self.ny = nx, ny
        self.glo, self.ghi = int(y0 > 0), int(y1 < ny)
        self.row_lo, self.row_hi = self.glo, self.glo + (y1 - y0)
        self.ny_local = self.row_hi + self.ghi
        self.y0 = y0
        self.s = state_global[:, y0 - self.glo:y1 + self.ghi].copy()
        self.halo_bytes = 4 * nx * 8
        self.prev = None

    def step(self, k):
        for _ in range(k):
            out = np.empty_like(self.s)
            ny, nx = self.ny_local, self.nx
            for i, (ex, ey) in enumerate(VEL):
                for y in range(ny):
                    for x in range(nx):
                        sx, sy = x - ex, y - ey
                        if 0 <= sx < nx and 0 <= sy < ny:
                            out[i, y, x] = self.s[i, sy, sx]
                        else:                      # bounce-back from the node itself
                            out[i, y, x] = self.s[OPPV[i], y, x]
            self.s = out

    def pack(self, p_lo, p_hi):
        if p_lo is not None:
            _buf(p_lo)[:] = self.s[DOWN, self.row_lo, :]
        if p_hi is not None:
            _buf(p_hi)[:] = self.s[UP, self.row_hi - 1, :]

    def unpack(self, p_lo, p_hi):
        if p_lo is not None:
            self.s[UP, 0, :] = _buf(p_lo)
        if p_hi is not None:
            self.s[DOWN, self.ny_local - 1, :] = _buf(p_hi)

    def interior(self):
        return self.s[:, self.row_lo:self.row_hi]

    def nusselt_sums(self):
        rows = self.interior()
        return float(rows[:, :, 0].sum()), float(rows[:, :, -1].sum())

    def residual_sums(self):
        cur = self.interior()[:3].sum(axis=2)
        prev = np.zeros_like(cur) if self.prev is None else self.prev
        self.prev = cur
        out = []
        for c in range(3):
            out += [float(((cur[c] - prev[c]) ** 2).sum()), float((cur[c] ** 2).sum())]
        return out + [0.0]


_BUFS = {}


def _buf(key):
    return _BUFS[key].reshape(4, -1)


def _make_buffer(nbytes):
    t = torch.zeros(nbytes // 8, dtype=torch.float64)
    _BUFS[t.data_ptr()] = t.numpy()
    return t


def _global_state(nx, ny, seed=5):
    return np.random.default_rng(seed).uniform(0.1, 1.0, size=(14, ny, nx))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _rank_main(rank, world, port, nx, ny, steps, out):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    import torch.distributed as dist
    from paper_2011_15073_gb300 import slabs
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        y0, y1 = slabs.partition(ny, world)[rank]
        ops = NumpySlab(nx, ny, y0, y1, _global_state(nx, ny))
        d = slabs.DistributedSlab(nx, ny, 1.0, 1e-2, 1e4, 6.2, ops=ops, make_buffer=_make_buffer)
        r0 = d.residual()
        d.step(steps)
        nu = d.nusselt()
        r1 = d.residual()
        out.put((rank, y0, y1, ops.interior().copy(), nu, r0, r1))
    finally:
        dist.destroy_process_group()


def _run(world, nx, ny, steps):
    import torch.multiprocessing as mp
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_rank_main, args=(r, world, port, nx, ny, steps, q)) for r in range(world)]
    for p in procs:
        p.start()
    res = sorted((q.get(timeout=180) for _ in procs), key=lambda t: t[0])
    for p in procs:
        p.join(timeout=60)
        assert p.exitcode == 0
    return res


@pytest.mark.parametrize("world,nx,ny", [(2, 7, 9), (3, 6, 11)])
def test_decomposed_streaming_equals_the_undivided_run(world, nx, ny):
    steps = 5
    res = _run(world, nx, ny, steps)
    whole = NumpySlab(nx, ny, 0, ny, _global_state(nx, ny))
    whole.residual_sums()
    whole.step(steps)
    got = np.concatenate([r[3] for r in res], axis=1)
    assert np.array_equal(got, whole.s)
    # Nu: the all-reduced sums over the interior rows, over ny
    h, c = whole.nusselt_sums()
    for r in res:
        assert r[4] == pytest.approx((h / ny, c / ny), rel=1e-14)
    # residual: the sums add up to the undivided run's
    wsums = whole.residual_sums()
    from paper_2011_15073_gb300 import slabs
    want = slabs.combine_residual(wsums)[0]
    assert all(r[6] == pytest.approx(want, rel=1e-12) for r in res)
    assert all(len({(r[1], r[2]) for r in res}) == world for _ in [0])


def test_partition_covers_the_rows_once():
    sys.path.insert(0, ROOT)
    from paper_2011_15073_gb300 import slabs
    for ny, parts in [(10, 3), (4096, 8), (5, 5), (7, 1)]:
        b = slabs.partition(ny, parts)
        assert b[0][0] == 0 and b[-1][1] == ny
        assert all(b[i][1] == b[i + 1][0] for i in range(parts - 1))
        sizes = [y1 - y0 for y0, y1 in b]
        assert max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        slabs.partition(3, 4)


def test_combine_residual():
    sys.path.insert(0, ROOT)
    from paper_2011_15073_gb300 import slabs
    r, nf = slabs.combine_residual([4.0, 16.0, 1.0, 100.0, 0.0, 0.0, 2.0])
    assert r == 0.5 and nf == 2.0
    assert slabs.combine_residual([np.inf, 1.0, 0, 1.0, 0, 1.0, 0])[0] == np.inf
