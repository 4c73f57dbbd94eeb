"""Host logic of the domain decomposition (CPU): the x-layer split, the
neighbour map, and the per-stage trace exchange between slab ranks with gloo
(world sizes 2 and 3, periodic and walled x).  The GPU side (pack kernel,
remote planes of the interface kernel, one-GPU slabs) is in test_gpu_partition.py."""
import os
import socket

import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

from paper_2605_16684_gb300 import decomp


def test_split_layers_cover_and_balance():
    for kx in (1, 2, 5, 7, 32, 33):
        for P in range(1, min(kx, 6) + 1):
            b = decomp.split_layers(kx, P)
            assert b[0][0] == 0 and b[-1][1] == kx
            assert all(x[1] == y[0] for x, y in zip(b, b[1:]))
            sizes = [e - s for s, e in b]
            assert min(sizes) >= 1 and max(sizes) - min(sizes) <= 1
    with pytest.raises(ValueError):
        decomp.split_layers(3, 4)


def test_neighbours():
    assert decomp.neighbours(0, 3, False) == (None, 1)
    assert decomp.neighbours(2, 3, False) == (1, None)
    assert decomp.neighbours(0, 3, True) == (2, 1)
    assert decomp.neighbours(2, 3, True) == (1, 0)
    assert decomp.neighbours(0, 2, True) == (1, 1)
    assert decomp.neighbours(0, 1, True) == (None, None)


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _trace(rank, which, n=37):
    # distinct contents per (rank, plane)
    return torch.arange(n, dtype=torch.float64) + 1000.0 * rank + (1.0 if which == "lo" else 2.0) / 4


def _rank(rank, world, port, periodic, directions, out):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        lo, hi = decomp.neighbours(rank, world, periodic)
        send_lo = _trace(rank, "lo") if lo is not None else None
        send_hi = _trace(rank, "hi") if hi is not None else None
        recv_lo = torch.full((37,), -1.0, dtype=torch.float64) if lo is not None else None
        recv_hi = torch.full((37,), -1.0, dtype=torch.float64) if hi is not None else None
        for k in range(3):  # several stages in a row
            if k == 1:
                # posted, other work while in flight, then waited for (Section 4.3)
                works = decomp.exchange_start(send_lo, send_hi, recv_lo, recv_hi, rank, world,
                                              periodic, directions=directions)
                busy = torch.arange(1000, dtype=torch.float64).sum()
                decomp.exchange_finish(works)
                assert float(busy) == 499500.0
            else:
                decomp.exchange(send_lo, send_hi, recv_lo, recv_hi, rank, world, periodic,
                                directions=directions)
        out[rank] = (None if recv_lo is None else recv_lo.tolist(),
                     None if recv_hi is None else recv_hi.tolist())
        dist.barrier()
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,periodic,directions", [(2, False, "both"), (2, True, "both"),
                                                       (3, True, "both"), (3, False, "up")])
def test_trace_exchange(world, periodic, directions):
    out = mp.get_context("spawn").Manager().dict()
    mp.start_processes(_rank, args=(world, _free_port(), periodic, directions, out),
                       nprocs=world, join=True, start_method="spawn")
    for r in range(world):
        lo, hi = decomp.neighbours(r, world, periodic)
        recv_lo, recv_hi = out[r]
        # the low plane receives the low neighbour's high trace, and vice versa
        if lo is None:
            assert recv_lo is None
        else:
            assert recv_lo == _trace(lo, "hi").tolist()
        if hi is None:
            assert recv_hi is None
        elif directions == "both":
            assert recv_hi == _trace(hi, "lo").tolist()
        else:
            assert recv_hi == [-1.0] * 37  # "up" moves only high-to-low-plane traces
