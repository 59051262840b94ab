"""Domain decomposition of the step, modelled on CPU ranks.

The grid is cut into y-slabs, one per rank (gloo, separate processes).  Each
step, every rank advances the cells of its own slab with the oracle, then
sends its two edge rows of all 16 S planes to the neighbouring ranks (the
radius-2 halo of the NND stencil) and receives theirs; periodic in y the ranks
form a ring, with outflow the end ranks use their own edge rows.  The
decomposed run must equal the monolithic oracle run bit for bit: the
per-cell arithmetic is the same, only the halo rows travel.  This is the
exchange a multi-GPU run would do (2 rows x nx x 16 S values per neighbour
and step); the GPU path itself runs as replicas on single-GPU machines.
"""
import os
import socket
import sys

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(bc_y):
    sys.path.insert(0, ROOT)
    from oracle import oracle as O
    from paper_2006_15932_gb300 import workloads as W

    pb = W.random_smooth(20, 18, 3, seed=41, reactive=True, force=True, bc=(W.OUTFLOW, bc_y))
    return pb, O.params_of(pb)


def _slabs(ny, world):
    cuts = [round(k * ny / world) for k in range(world + 1)]
    return [(cuts[k], cuts[k + 1]) for k in range(world)]


def _worker(rank, world, port, bc_y, nsteps, q):
    sys.path.insert(0, ROOT)
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        from oracle import oracle as O

        pb, p = _problem(bc_y)
        periodic = bc_y == 0
        f = O.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T)  # every rank starts from the same field
        y0, y1 = _slabs(pb.ny, world)[rank]
        up, down = (rank + 1) % world, (rank - 1) % world
        has_up = periodic or rank + 1 < world
        has_down = periodic or rank > 0
        status = 0
        for _ in range(nsteps):
            slab, st = O.step_region(p, f, 0, pb.nx, y0, y1)
            status |= st
            f[:, :, y0:y1, :] = slab
            # halo exchange: my two top rows go up, my two bottom rows go down
            reqs = []
            top = torch.from_numpy(np.ascontiguousarray(f[:, :, y1 - 2:y1, :]))
            bot = torch.from_numpy(np.ascontiguousarray(f[:, :, y0:y0 + 2, :]))
            from_down = torch.empty_like(top)
            from_up = torch.empty_like(bot)
            if has_up:
                reqs.append(dist.isend(top, up, tag=1))
                reqs.append(dist.irecv(from_up, up, tag=2))
            if has_down:
                reqs.append(dist.isend(bot, down, tag=2))
                reqs.append(dist.irecv(from_down, down, tag=1))
            for r in reqs:
                r.wait()
            if has_up:
                rows = [(y1 + k) % pb.ny for k in range(2)]
                f[:, :, rows, :] = from_up.numpy()
            if has_down:
                rows = [(y0 - 2 + k) % pb.ny for k in range(2)]
                f[:, :, rows, :] = from_down.numpy()
        ref, st_ref = O.run(p, O.init_feq(p, pb.rho_s, pb.ux, pb.uy, pb.T), nsteps)
        same = bool(np.array_equal(f[:, :, y0:y1, :], ref[:, :, y0:y1, :]))
        q.put((rank, same, status, st_ref))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,bc_y", [(3, 0), (2, 1)])
def test_y_slab_decomposition_matches_monolithic_bitwise(world, bc_y):
    from oracle import oracle as O

    O.build()
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_worker, args=(r, world, port, bc_y, 12, q)) for r in range(world)]
    for p in procs:
        p.start()
    for p in procs:
        p.join(180)
        assert p.exitcode == 0
    got = sorted(q.get(timeout=10) for _ in range(world))
    for rank, same, status, st_ref in got:
        assert status == 0 and st_ref == 0
        assert same, f"rank {rank}: decomposed slab differs from the monolithic run"
