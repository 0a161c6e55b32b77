"""Row-strip decomposition of one image over CPU ranks (gloo): each rank steps its strip plus a 6-row halo that
it exchanges with its neighbours once per iteration, and the strips put together equal the single-domain solve of
the oracle.  The step on each extended strip is the oracle's own iPiano step."""
import functools
import os
import socket

import numpy as np
import pytest
import torch
import torch.distributed as dist
import torch.multiprocessing as mp

import oracle as O
from paper_1609_05722_gb300 import domain, synth

H, W, ITERS, GAMMA = 40, 23, 4, 0.8


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _problem(h, model, bc, tau):
    k, a = synth.filter_bank()
    return O.Problem(k, a, h, W, bc=bc, model=model, lam=1.0, tau=tau, gamma=GAMMA, nthreads=1)


def _data(model):
    y = synth.poisson_observation(synth.clean_image(H, W, 77), 4.0, 78)
    d = y if model == O.MODEL_DIRECT else O.anscombe(y)
    u0 = np.maximum(d, 0.5) if model == O.MODEL_DIRECT else d.copy()
    return d, u0


@functools.lru_cache(maxsize=None)
def _tau(bc):
    k, a = synth.filter_bank()
    return 0.99 * 2 * (1 - GAMMA) / (O.lipschitz(k, a, bc, 512) + 2e-3)


def _worker(rank, world, port, model, bc, tau, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world)
    try:
        e0, e1 = domain.extended_rows(H, world, rank)
        d, u0 = _data(model)
        pr = _problem(e1 - e0, model, bc, tau)

        def step(d_ext, u, u_prev):
            return torch.from_numpy(pr.step(d_ext.numpy(), u.numpy(), u_prev.numpy()))

        own = domain.solve_strip(step, torch.from_numpy(d[e0:e1].copy()), torch.from_numpy(u0[e0:e1].copy()),
                                 ITERS, H, world, rank, dist)
        q.put((rank, own.numpy()))
    finally:
        dist.destroy_process_group()


@pytest.mark.parametrize("world,model,bc", [(2, O.MODEL_ANS_L2, O.BC_SYMMETRIC), (3, O.MODEL_DIRECT, O.BC_SYMMETRIC),
                                            (3, O.MODEL_ANS_L2, O.BC_ZERO)])
def test_strips_equal_the_single_domain_solve(world, model, bc):
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    tau = _tau(bc)
    procs = [ctx.Process(target=_worker, args=(r, world, port, model, bc, tau, q)) for r in range(world)]
    for p in procs:
        p.start()
    parts = dict(q.get(timeout=240) for _ in range(world))
    for p in procs:
        p.join(60)
        assert p.exitcode == 0
    got = np.concatenate([parts[r] for r in range(world)])
    d, u0 = _data(model)
    pr = _problem(H, model, bc, tau)
    u, up = u0.copy(), u0.copy()
    for _ in range(ITERS):
        u, up = pr.step(d, u, up), u
    assert got.shape == u.shape
    # the same FP64 operations in the same order for every owned pixel
    np.testing.assert_allclose(got, u, rtol=0, atol=1e-12 * np.abs(u).max())
    # negative control: strips whose halo rows keep their initial values (no exchange) miss the solve next to a
    # cut by far more than rounding
    stale = []
    for r in range(world):
        (r0, r1), (e0, e1) = domain.strip_rows(H, world, r), domain.extended_rows(H, world, r)
        ps = _problem(e1 - e0, model, bc, tau)
        us, ups = u0[e0:e1].copy(), u0[e0:e1].copy()
        for _ in range(ITERS):
            un = ps.step(d[e0:e1], us, ups)
            ups[r0 - e0:r1 - e0], us[r0 - e0:r1 - e0] = us[r0 - e0:r1 - e0], un[r0 - e0:r1 - e0]
        stale.append(us[r0 - e0:r1 - e0])
    assert np.abs(np.concatenate(stale) - u).max() > 1e3 * 1e-12 * np.abs(u).max()


def test_strip_partition():
    for h, world in [(40, 2), (41, 3), (12, 2), (1000, 7)]:
        rows = [domain.strip_rows(h, world, r) for r in range(world)]
        assert rows[0][0] == 0 and rows[-1][1] == h
        assert all(a[1] == b[0] for a, b in zip(rows, rows[1:]))
        sizes = [r1 - r0 for r0, r1 in rows]
        assert max(sizes) - min(sizes) <= 1 and min(sizes) >= domain.HALO
        for r in range(world):
            e0, e1 = domain.extended_rows(h, world, r)
            assert e0 == max(0, rows[r][0] - domain.HALO) and e1 == min(h, rows[r][1] + domain.HALO)
    with pytest.raises(ValueError):
        domain.strip_rows(11, 2, 0)
    with pytest.raises(ValueError):
        domain.strip_rows(40, 2, 2)


def _dying_worker(rank, world, port, q):
    import datetime
    import time
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    dist.init_process_group("gloo", rank=rank, world_size=world, timeout=datetime.timedelta(seconds=10))
    if rank == 1:
        os._exit(3)  # this rank leaves between steps, before its first exchange
    d = torch.zeros((H, W), dtype=torch.float64)
    e0, e1 = domain.extended_rows(H, world, rank)
    t0 = time.time()
    try:
        domain.solve_strip(lambda d_, u, up: u, d[e0:e1], d[e0:e1], 3, H, world, rank, dist)
        q.put((rank, "finished", time.time() - t0))
    except Exception as e:  # the exchange with the lost neighbour fails instead of waiting forever
        q.put((rank, type(e).__name__, time.time() - t0))
    # os._exit skips the queue's feeder thread: flush the message before leaving
    q.close()
    q.join_thread()
    os._exit(0)


def test_a_lost_neighbour_ends_the_exchange_with_an_error():
    ctx = mp.get_context("spawn")
    q = ctx.Queue()
    port = _free_port()
    procs = [ctx.Process(target=_dying_worker, args=(r, 2, port, q)) for r in range(2)]
    for p in procs:
        p.start()
    rank, what, elapsed = q.get(timeout=120)
    for p in procs:
        p.join(60)
    assert rank == 0 and what != "finished" and elapsed < 60
    assert procs[1].exitcode == 3 and procs[0].exitcode == 0
