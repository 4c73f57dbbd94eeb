"""Domain decomposition along x (Section 4.3: one process per GPU, element
partitions, face traces exchanged every stage).

A mesh is cut into slabs of whole x element layers; slab r is a handle created
with es_dg_create_partition whose cut x planes take their outside state from a
trace received from the neighbouring slab.  All slabs on one GPU are stepped by
the library itself (`_lib.PartitionedSolver`, device-to-device copies).  Across
processes, `DistributedSlab` runs one slab per rank and moves the traces with
torch.distributed point-to-point messages (NCCL between GPUs, gloo on CPU) before
every stage: pack (kernel), exchange posted, the interface kernel on the faces
that need no trace while the messages are in flight (Section 4.3's overlap), the
faces of the cut planes once they have landed, volume kernel with the RK
update.  The exchange is the only communication; there is no collective on the
data path.
"""
from __future__ import annotations

from typing import List, Optional, Tuple


def split_layers(kx: int, P: int) -> List[Tuple[int, int]]:
    """P contiguous ranges of x element layers covering 0..kx, sizes differing by
    at most one (the first kx % P ranges one layer longer)."""
    if not (1 <= P <= kx):
        raise ValueError("need 1 <= P <= kx")
    base, extra = divmod(kx, P)
    out, b = [], 0
    for r in range(P):
        e = b + base + (1 if r < extra else 0)
        out.append((b, e))
        b = e
    return out


def neighbours(rank: int, world: int, periodic: bool) -> Tuple[Optional[int], Optional[int]]:
    """Ranks across the low and high x planes of slab `rank` (None at a wall)."""
    lo = rank - 1 if rank > 0 else (world - 1 if periodic and world > 1 else None)
    hi = rank + 1 if rank + 1 < world else (0 if periodic and world > 1 else None)
    return lo, hi


# message tags: a slab's high trace becomes its high neighbour's low trace and
# vice versa (two messages between the same pair when world = 2 and x is periodic)
TAG_TO_LO_PLANE, TAG_TO_HI_PLANE = 11, 12


def exchange(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, periodic: bool,
             group=None, directions: str = "both") -> None:
    """Move one stage's traces between neighbouring slabs with torch.distributed.

    send_hi of rank r lands in recv_lo of its high neighbour; send_lo in recv_hi of
    its low neighbour.  directions="up" moves only the high-to-low-plane half (the
    face geometry hand-over).  Tensors of a plane without a neighbour may be None.
    Blocks until every message of this rank has completed."""
    exchange_finish(exchange_start(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic,
                                   group, directions))


def exchange_finish(works) -> None:
    """Wait for the messages posted by exchange_start."""
    for w in works:
        w.wait()


def exchange_start(send_lo, send_hi, recv_lo, recv_hi, rank: int, world: int, periodic: bool,
                   group=None, directions: str = "both") -> list:
    """Post one stage's trace messages (as exchange) and return their handles
    without waiting: work that needs no trace can run while they are in flight
    (Section 4.3), and exchange_finish waits for them."""
    import torch.distributed as dist
    lo, hi = neighbours(rank, world, periodic)
    ops = []
    # issue order is the same on every rank (sends before receives, high plane
    # first), which also fixes the matching where a transport ignores tags
    if hi is not None:
        ops.append(dist.P2POp(dist.isend, send_hi, hi, group, TAG_TO_LO_PLANE))
    if lo is not None and directions == "both":
        ops.append(dist.P2POp(dist.isend, send_lo, lo, group, TAG_TO_HI_PLANE))
    if lo is not None:
        ops.append(dist.P2POp(dist.irecv, recv_lo, lo, group, TAG_TO_LO_PLANE))
    if hi is not None and directions == "both":
        ops.append(dist.P2POp(dist.irecv, recv_hi, hi, group, TAG_TO_HI_PLANE))
    return dist.batch_isend_irecv(ops) if ops else []


class DistributedSlab:
    """This rank's slab of a mesh split along x over the process group: a
    partition handle on this process's GPU plus its four trace buffers.

    Not exercised on more than one GPU here (one GPU per machine in this
    environment); the single-GPU slabs (`_lib.PartitionedSolver`) run the same
    pack / exchange / stage sequence inside the library, and the exchange itself
    is tested with gloo ranks on CPU."""

    def __init__(self, kx, ky, kz, N, rank: int, world: int, periodic=(1, 1, 0), group=None,
                 **kw):
        import torch
        from ._lib import Solver
        self.rank, self.world, self.group = rank, world, group
        self.periodic_x = bool(periodic[0])
        self.bounds = split_layers(kx, world)[rank]
        self.s = Solver(kx, ky, kz, N, periodic=periodic, part=self.bounds, **kw)
        _, _, remote, n = self.s.partition_info()
        self.t = [torch.zeros(n, dtype=torch.float64, device="cuda") if remote[k % 2] else None
                  for k in range(4)]  # send_lo, send_hi, recv_lo, recv_hi
        self.s.set_traces(*self.t)

    def _exchange(self, directions="both"):
        self._exchange_finish(self._exchange_start(directions))

    def _exchange_start(self, directions="both"):
        import torch
        torch.cuda.current_stream().wait_stream(self.s.stream)  # the traces are packed
        return exchange_start(*self.t, self.rank, self.world, self.periodic_x, self.group,
                              directions)

    def _exchange_finish(self, works):
        import torch
        exchange_finish(works)
        self.s.stream.wait_stream(torch.cuda.current_stream())  # the traces have landed

    def connect(self):
        """Hand the high planes' face geometry to the high neighbours (once)."""
        self.s.pack_traces(geometry=True)
        self._exchange("up")
        self.s.accept_geometry_trace()
        self.s.sync()

    def step(self, dt: float, nsteps: int = 1):
        """LSRK steps with Section 4.3's overlap: the faces that need no trace run
        while the stage's traces are in flight, those of the cut planes after."""
        for _ in range(nsteps):
            for stage in range(5):
                self.s.pack_traces()
                works = self._exchange_start()
                self.s.launch(3, stage, dt)  # interface fluxes that need no trace
                self._exchange_finish(works)
                self.s.launch(4, stage, dt)  # those of the cut planes, with the traces
                self.s.launch(2, stage, dt)  # volume, lifts, source and the RK update
