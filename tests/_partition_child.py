"""One rank of a gloo process group (started by torchrun from
tests/test_partition.py): builds its send buffer of the partitioned transform
from a seeded global Delta in the layout include/sht.h documents, exchanges it
with sht.exchange, and checks that its receive buffer holds every order of
its rings in the documented receive layout."""
import json
import os
import sys

import numpy as np
import torch
import torch.distributed as dist

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
sys.path.insert(0, ROOT)

from paper_1010_1260_gb300 import sht  # noqa: E402


def main():
    dist.init_process_group("gloo")
    rank, world = dist.get_rank(), dist.get_world_size()
    lmax = mmax = 21
    nphi = np.array([4 * i for i in range(1, 6)] + [24] * 11 + [4 * i for i in range(5, 0, -1)], dtype=np.int32)
    nrings, B = len(nphi), 3
    mo, ro = sht.partition(lmax, mmax, nphi, world)
    rng = np.random.default_rng(9)
    delta = rng.standard_normal((B, nrings, mmax + 1)) + 1j * rng.standard_normal((B, nrings, mmax + 1))
    mine_m = np.flatnonzero(mo == rank)
    # send: for each destination q, q's rings x maps x this rank's orders
    send = np.concatenate([delta[:, ro == q][:, :, mine_m].transpose(1, 0, 2).reshape(-1) for q in range(world)])
    recv = sht.exchange(torch.from_numpy(send), mo, ro, B).numpy()
    # receive: for each source p, this rank's rings x maps x p's orders
    rings = np.flatnonzero(ro == rank)
    got = np.full((B, len(rings), mmax + 1), np.nan + 0j)
    off = 0
    for p in range(world):
        ms = np.flatnonzero(mo == p)
        blk = recv[off: off + len(rings) * B * len(ms)].reshape(len(rings), B, len(ms))
        got[:, :, ms] = blk.transpose(1, 0, 2)
        off += blk.size
    ok = bool(off == recv.size and np.array_equal(got, delta[:, rings]))
    every = [None] * world
    dist.all_gather_object(every, {"rank": rank, "ok": ok, "rings": len(rings), "orders": int(len(mine_m))})
    dist.barrier()
    dist.destroy_process_group()
    if rank == 0:
        print(json.dumps({"world": world, "ranks": every}), flush=True)


if __name__ == "__main__":
    main()
