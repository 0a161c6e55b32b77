"""Row-strip decomposition with the CUDA step: 2 and 3 gloo ranks, one GPU.

Each rank steps its extended strip (its rows plus the 6-row halo exchanged before every step) with the library's
FP32 step (foe_ipiano_step through the C ABI), and the strips put together must equal, bit for bit, the same CUDA
step run on the whole image (the FP32 kernel's arithmetic at a pixel does not depend on where its tile starts),
and the FP64 oracle's single-domain solve within the FP32 bound.  The ranks exchange host
tensors over gloo between steps; no kernel of one rank waits on another rank.

The iterate crosses the exchange as FP64 values u = u_hi + u_lo (the FP32 pair of the plain FP32 path), so no
precision is lost at the strip seams: the per-pixel arithmetic of an owned pixel is that of the single-domain
step, whatever the strip's tiling.
"""
import os
import socket

import numpy as np
import pytest

torch = pytest.importorskip("torch")
import torch.distributed as dist  # noqa: E402
import torch.multiprocessing as mp  # noqa: E402

import oracle as O  # noqa: E402
from paper_1609_05722_gb300 import build as B  # noqa: E402
from paper_1609_05722_gb300 import domain, synth  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402

pytestmark = pytest.mark.gpu

H, W, ITERS = 96, 70, 20
GAMMA = float(np.float32(0.8))


def _free_port():
    with socket.socket() as s:
        s.bind(("127.0.0.1", 0))
        return s.getsockname()[1]


def _data(model):
    y = synth.poisson_observation(synth.clean_image(H, W, 31), 4.0, 32)
    return O.anscombe(y) if model != F.FOE_MODEL_DIRECT else y.astype(np.float64)


class CudaStep:
    """step(d, u, u_prev) -> u_next on an h x W strip (FP64 host tensors), by one launch of the FP32 step kernel:
    u_hi = fl32(u), u_lo = fl32(u - u_hi), delta = fl32(u - u_prev)."""

    def __init__(self, ctx, h, model, tau, bc):
        self.ctx, self.h, self.model, self.tau, self.bc = ctx, h, model, tau, bc
        self.ld = (W + 3) // 4 * 4

    def _dev(self, a):
        t = torch.zeros((self.h, self.ld), dtype=torch.float32, device="cuda")
        t[:, :W] = a.to(torch.float32).cuda()
        return t

    def __call__(self, d, u, u_prev):
        hi = u.to(torch.float32)
        lo = (u - hi.double()).to(torch.float32)
        dl = (u - u_prev).to(torch.float32)
        uh, ul, dd, de = self._dev(hi), self._dev(lo), self._dev(d), self._dev(dl)
        un = torch.zeros_like(uh)
        F.foe_ipiano_step(self.ctx, uh, ul, de, dd, un, self.h, W, self.ld, self.model, 1.0, self.tau, GAMMA,
                          self.bc, F.FOE_PREC_FP32)
        torch.cuda.synchronize()
        return un[:, :W].double().cpu() + ul[:, :W].double().cpu()


def _ctx():
    k, a = synth.filter_bank()
    return F.foe_create(k.astype(np.float32), a.astype(np.float32))


def _worker(rank, world, port, model, bc, tau, q):
    os.environ.update(MASTER_ADDR="127.0.0.1", MASTER_PORT=str(port), RANK=str(rank), WORLD_SIZE=str(world))
    torch.cuda.set_device(0)
    dist.init_process_group("gloo", rank=rank, world_size=world)
    ctx = _ctx()
    try:
        e0, e1 = domain.extended_rows(H, world, rank)
        d = torch.from_numpy(_data(model)[e0:e1].copy())
        own = domain.solve_strip(CudaStep(ctx, e1 - e0, model, tau, bc), d, d.clone(), ITERS, H, world, rank, dist)
        q.put((rank, own.numpy()))
    finally:
        F.foe_destroy(ctx)
        dist.destroy_process_group()


@pytest.mark.parametrize("world,model,bc", [(2, F.FOE_MODEL_ANS_L2, F.FOE_BC_SYMMETRIC),
                                            (3, F.FOE_MODEL_ANS_IDIV, F.FOE_BC_SYMMETRIC),
                                            (3, F.FOE_MODEL_ANS_L2, F.FOE_BC_ZERO)])
def test_strips_with_the_cuda_step_equal_the_single_domain_solve(world, model, bc):
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    ctx = _ctx()
    tau, _ = F.foe_step_size(ctx, bc, GAMMA)
    try:
        mpc = mp.get_context("spawn")
        q = mpc.Queue()
        port = _free_port()
        procs = [mpc.Process(target=_worker, args=(r, world, port, model, bc, tau, q)) for r in range(world)]
        for p in procs:
            p.start()
        parts = dict(q.get(timeout=300) for _ in range(world))
        for p in procs:
            p.join(60)
            assert p.exitcode == 0
        got = np.concatenate([parts[r] for r in range(world)])
        # the same CUDA step on the whole image
        d = torch.from_numpy(_data(model))
        step = CudaStep(ctx, H, model, tau, bc)
        u, up = d.clone(), d.clone()
        for _ in range(ITERS):
            up, u = u, step(d, u, up)
        ref_gpu = u.numpy()
    finally:
        F.foe_destroy(ctx)
    scale = np.abs(ref_gpu).max()
    print(f"strips world={world} model={model} bc={bc}: max |strips - whole| {np.abs(got - ref_gpu).max():.3e} "
          f"(bitwise {np.array_equal(got, ref_gpu)})")
    assert np.array_equal(got, ref_gpu)
    # and the oracle's single-domain solve (FP64) within the FP32 path's bound
    k, a = synth.filter_bank()
    pr = O.Problem(k.astype(np.float32).astype(np.float64), a.astype(np.float32).astype(np.float64), H, W, bc=bc,
                   model=model, lam=1.0, tau=tau, gamma=GAMMA)
    dd = _data(model)
    uo, _ = pr.ipiano(dd, dd, dd, ITERS)
    assert np.abs(got - uo).max() <= 2e-5 * scale
