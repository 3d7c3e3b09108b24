"""Slab decomposition of one grid over several devices, with one halo exchange per pass.

The paper names distribution over several devices as the motivation for its blocking and as
future work (arXiv 1802.00438, Sec. 1 and 8).  The overlapped-tile argument of Sec. 3.2 carries
over unchanged to a split between devices: a rank that holds its own rows plus `halo` rows of
each neighbour can advance `halo` steps on its own, because a wrong value at the cut (the cut
is clamped like a domain edge) travels inward by one row per step and never reaches the rows it
owns.  So the grid is cut along its slowest axis (y in 2D, z in 3D) into slabs of whole rows or
planes, and every pass of T = halo steps is

    1. exchange: each rank sends its first `halo` owned rows to the rank before it and its last
       `halo` owned rows to the rank after it, receiving the neighbours' rows into its halo;
    2. compute: the rank advances its extended slab (owned rows plus halos) by up to T steps
       with the engine's own temporally-blocked plan; the owned rows are exact.

Exchanges go device to device: torch.distributed point-to-point (NCCL on GPUs; gloo runs the
same schedule on host tensors) or, for slabs held by one process, plain copies into the
receiving slab's own buffer.  Nothing reads another device's memory directly (no peer loads,
no multicast): a halo is always copied into the receiver's memory first.

Arrays are (ny, nx) for 2D and (nz, ny, nx) for 3D, rows (planes) along axis 0.
"""
from __future__ import annotations

from dataclasses import dataclass


def partition(n: int, parts: int):
    """Balanced contiguous split of n rows into `parts` ranges [(lo, hi), ...], every part
    non-empty (parts <= n)."""
    if parts < 1 or parts > n:
        raise ValueError(f"cannot split {n} rows into {parts} non-empty slabs")
    base, extra = divmod(n, parts)
    out, lo = [], 0
    for r in range(parts):
        hi = lo + base + (1 if r < extra else 0)
        out.append((lo, hi))
        lo = hi
    return out


@dataclass
class Slab:
    """One rank's part of the grid: it owns rows [lo, hi) and holds rows [ext_lo, ext_hi)."""
    rank: int
    parts: int
    n: int          # rows of the whole grid
    lo: int
    hi: int
    halo: int

    @property
    def ext_lo(self) -> int:
        return max(0, self.lo - self.halo)

    @property
    def ext_hi(self) -> int:
        return min(self.n, self.hi + self.halo)

    @property
    def ext_rows(self) -> int:
        return self.ext_hi - self.ext_lo

    # row ranges in the extended slab's own indexing
    def own(self):
        return self.lo - self.ext_lo, self.hi - self.ext_lo

    def top_halo(self):          # rows above the owned ones (from rank - 1)
        return 0, self.lo - self.ext_lo

    def bottom_halo(self):       # rows below the owned ones (from rank + 1)
        return self.hi - self.ext_lo, self.ext_rows

    def send_up(self):           # my first halo rows, for rank - 1's bottom halo
        a, _ = self.own()
        return a, a + min(self.halo, self.hi - self.lo)

    def send_down(self):         # my last halo rows, for rank + 1's top halo
        _, b = self.own()
        return b - min(self.halo, self.hi - self.lo), b


def slabs(n: int, parts: int, halo: int):
    """The slabs of an n-row grid over `parts` ranks with halos of `halo` rows.  Each slab must
    own at least `halo` rows, so that a neighbour's halo comes from one rank."""
    if halo < 1:
        raise ValueError("halo must be at least one row")
    out = [Slab(r, parts, n, lo, hi, halo) for r, (lo, hi) in enumerate(partition(n, parts))]
    if parts > 1 and min(s.hi - s.lo for s in out) < halo:
        raise ValueError(f"slabs of {n // parts} rows are thinner than the halo ({halo} rows)")
    return out


def scatter(full, sl: Slab):
    """The extended slab of a whole-grid array (a view)."""
    return full[sl.ext_lo:sl.ext_hi]


def passes(steps: int, T: int):
    """Steps of each pass: T, ..., T, remainder (Eq. 8 with the remainder of Sec. 3.2)."""
    out = [T] * (steps // T)
    if steps % T:
        out.append(steps % T)
    return out


class LocalExchange:
    """Halo exchange between slabs held by one process (one device or several): copies of the
    sender's boundary rows into the receiver's own halo rows (torch tensors or numpy arrays)."""

    def __init__(self, slab_list):
        self.slabs = slab_list

    def __call__(self, grids):
        """grids[r]: extended slab array of rank r, updated in place."""
        for r in range(len(self.slabs) - 1):
            a, b = self.slabs[r], self.slabs[r + 1]
            s0, s1 = a.send_down()          # rank r's last owned rows -> rank r+1's top halo
            t0, t1 = b.top_halo()
            grids[r + 1][t0:t1] = grids[r][s0:s1]
            s0, s1 = b.send_up()            # rank r+1's first owned rows -> rank r's bottom halo
            t0, t1 = a.bottom_halo()
            grids[r][t0:t1] = grids[r + 1][s0:s1]


class DistExchange:
    """Halo exchange between ranks of a torch.distributed process group: non-blocking sends of
    the boundary rows and receives into the halo rows (contiguous row blocks), all completed
    before the pass starts.  The grid tensor lives on the rank's device (NCCL) or the host
    (gloo)."""

    def __init__(self, slab: Slab, dist, group=None):
        self.slab = slab
        self.dist = dist
        self.group = group

    def __call__(self, grid):
        sl, dist = self.slab, self.dist
        if not grid.is_contiguous():
            raise ValueError("the slab must be a contiguous array of rows")
        reqs = []
        if sl.rank > 0:
            a, b = sl.send_up()
            reqs.append(dist.isend(grid[a:b], sl.rank - 1, group=self.group, tag=1))
            a, b = sl.top_halo()
            reqs.append(dist.irecv(grid[a:b], sl.rank - 1, group=self.group, tag=2))
        if sl.rank < sl.parts - 1:
            a, b = sl.send_down()
            reqs.append(dist.isend(grid[a:b], sl.rank + 1, group=self.group, tag=2))
            a, b = sl.bottom_halo()
            reqs.append(dist.irecv(grid[a:b], sl.rank + 1, group=self.group, tag=1))
        for q in reqs:
            q.wait()


def run_slab(sl: Slab, grid, steps: int, T: int, advance, exchange):
    """Advance one rank's extended slab `grid` by `steps` steps: per pass one halo exchange,
    then advance(grid, ts) for ts <= T steps.  advance must update the extended slab in place
    (clamping at its own edges, as the engine's plans do); exchange(grid) fills the halo rows.
    Returns grid; its owned rows hold the result."""
    if T > sl.halo:
        raise ValueError("a pass may fuse at most `halo` steps")
    for ts in passes(steps, T):
        if sl.parts > 1:
            exchange(grid)
        advance(grid, ts)
    return grid


def run_local(slab_list, grids, steps: int, T: int, advance):
    """All slabs in one process: per pass one LocalExchange, then advance(r, grids[r], ts) for
    every rank r."""
    ex = LocalExchange(slab_list)
    for ts in passes(steps, T):
        if len(slab_list) > 1:
            ex(grids)
        for r in range(len(slab_list)):
            advance(r, grids[r], ts)
    return grids


class PlanAdvance:
    """advance() for one rank's slab on its CUDA device: an engine plan sized to the extended
    slab, run in place (the plan keeps its own ping-pong scratch)."""

    def __init__(self, st, kind, ndim, sl: Slab, nx, ny, nz=1, coeffs=None, power=None,
                 **plan_kw):
        self.st = st
        if ndim == 2:
            self.shape = (sl.ext_rows, nx)
            self.plan = st.Plan(kind, 2, nx, sl.ext_rows, **plan_kw)
        else:
            self.shape = (sl.ext_rows, ny, nx)
            self.plan = st.Plan(kind, 3, nx, ny, sl.ext_rows, **plan_kw)
        self.coeffs = coeffs
        self.power = power

    def __call__(self, grid, ts):
        self.plan.run(grid, grid, self.coeffs, ts, power=self.power)

    def close(self):
        self.plan.close()
