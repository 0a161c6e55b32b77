"""Continuous-batching server: results, admission under the HBM budget, alone vs in the mix.

Each tile of each image is computed by the same kernel code from the same inputs whatever else is in
the launch, so a request's result must be bit-for-bit the same served alone, served in a mix that
changes every tick, and computed by foe_denoise.
"""
import numpy as np
import pytest

torch = pytest.importorskip("torch")

from paper_1609_05722_gb300 import build as B  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402
from paper_1609_05722_gb300 import synth  # noqa: E402

pytestmark = pytest.mark.gpu

# (H, W, peak, iters)
REQS = [(64, 64, 4.0, 30), (100, 37, 12.0, 20), (128, 200, 2.0, 45), (33, 90, 30.0, 10), (75, 75, 1.0, 0),
        (160, 128, 6.0, 25)]


@pytest.fixture(scope="module")
def ctx():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    torch.cuda.set_device(0)
    k, a = synth.filter_bank()
    c = F.foe_create(k.astype(np.float32), a.astype(np.float32))
    yield c
    F.foe_destroy(c)


def images():
    out = []
    for j, (H, W, peak, it) in enumerate(REQS):
        y = synth.poisson_observation(synth.clean_image(H, W, 900 + j), peak, 950 + j).astype(np.float32)
        out.append(torch.from_numpy(y).pin_memory())
    return out


def reference(ctx, ys, prec):
    refs = []
    for (H, W, peak, it), y in zip(REQS, ys):
        ld = (W + 3) // 4 * 4
        yd = torch.zeros((H, ld), dtype=torch.float32, device="cuda")
        yd[:, :W] = y.cuda()
        xd = torch.zeros_like(yd)
        F.foe_denoise(ctx, yd, xd, H, W, ld, peak, F.SolveOpts(model=F.FOE_MODEL_AUTO, iters=it, prec=prec))
        refs.append(xd[:, :W].cpu().numpy())
    torch.cuda.synchronize()
    return refs


def serve(ctx, ys, order_ticks, prec, budget, max_active, per_tick, graphs):
    """order_ticks: list of (request index, tick at which it is submitted)."""
    srv = F.foe_server_create(ctx, budget, max_active, per_tick, graphs,
                              F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=prec))
    outs = {j: torch.full((REQS[j][0], REQS[j][1]), float("nan")).pin_memory() for j, _ in order_ticks}
    ids = {}
    tick = 0
    max_active_seen, max_bytes = 0, 0
    try:
        while True:
            for j, t in order_ticks:
                if t == tick:
                    H, W, peak, it = REQS[j]
                    ids[F.foe_server_submit(srv, ys[j], outs[j], H, W, peak, it, ctx=ctx)] = j
            F.foe_server_tick(srv, ctx)
            st = F.foe_server_get_stats(srv)
            max_active_seen = max(max_active_seen, st["active"])
            max_bytes = max(max_bytes, st["bytes_in_use"])
            assert st["bytes_in_use"] <= st["bytes_budget"]
            tick += 1
            if st["completed"] == len(order_ticks) and tick > max(t for _, t in order_ticks):
                break
            assert tick < 1000
        done = F.foe_server_poll(srv)
        assert sorted(done) == sorted(ids)
    finally:
        F.foe_server_destroy(srv)
    return {j: outs[j].numpy() for j in outs}, max_active_seen, max_bytes


@pytest.mark.parametrize("prec", [F.FOE_PREC_FP32, F.FOE_PREC_BF16])
@pytest.mark.parametrize("graphs", [True, False])
def test_mix_equals_alone_equals_denoise(ctx, prec, graphs):
    ys = images()
    refs = reference(ctx, ys, prec)
    # staggered arrivals, small slot count: the batch changes every tick
    mix, _, _ = serve(ctx, ys, [(0, 0), (1, 0), (2, 1), (3, 3), (4, 4), (5, 6)], prec, 64 << 20, 3, 7, graphs)
    for j in mix:
        alone, _, _ = serve(ctx, ys, [(j, 0)], prec, 64 << 20, 1, 7, graphs)
        assert np.array_equal(alone[j], refs[j]), j
        assert np.array_equal(mix[j], refs[j]), j


def test_admission_respects_budget_and_slots(ctx):
    ys = images()
    # budget for about two of the larger requests' state (5 planes of H x ld FP32)
    need = [5 * H * ((W + 3) // 4 * 4) * 4 for H, W, _, _ in REQS]
    budget = max(1 << 20, sorted(need)[-1] + sorted(need)[-2] + 4096)
    out, max_active, max_bytes = serve(ctx, ys, [(j, 0) for j in range(len(REQS))], F.FOE_PREC_BF16, budget, 4, 5,
                                       True)
    assert max_active <= 4 and max_bytes <= budget
    refs = reference(ctx, ys, F.FOE_PREC_BF16)
    for j in out:
        assert np.array_equal(out[j], refs[j])


def test_request_larger_than_budget_is_refused(ctx):
    srv = F.foe_server_create(ctx, 1 << 20, 4, 5, True, F.SolveOpts())
    try:
        y = np.zeros((512, 512), np.float32)
        with pytest.raises(F.FoeError) as e:
            F.foe_server_submit(srv, y, y, 512, 512, 4.0, 10, ctx=ctx)
        assert e.value.status == F.FOE_ENOMEM
    finally:
        F.foe_server_destroy(srv)


def test_expired_device_wait_stops_the_server(ctx):
    """A bounded device wait made to expire (one withheld mbarrier arrival, no GPU fault): the tick that completes
    the affected round reports FOE_ETIMEOUT, every later tick returns it without device work, no affected request
    is reported, and after foe_device_status a new server on the same context serves bit-exact results."""
    ys = images()
    srv = F.foe_server_create(ctx, 64 << 20, 4, 5, True, F.SolveOpts(model=F.FOE_MODEL_AUTO, prec=F.FOE_PREC_BF16))
    outs = [torch.zeros((H, W)).pin_memory() for H, W, _, _ in REQS]
    try:
        for j in (0, 2):
            H, W, peak, it = REQS[j]
            F.foe_server_submit(srv, ys[j], outs[j], H, W, peak, it, ctx=ctx)
        F.foe_debug_withhold_arrival(ctx)
        F.foe_server_tick(srv, ctx)                      # queues the affected round
        with pytest.raises(F.FoeError) as e:
            for _ in range(3):
                F.foe_server_tick(srv, ctx)              # completes it
        assert e.value.status == F.FOE_ETIMEOUT
        with pytest.raises(F.FoeError) as e:
            F.foe_server_tick(srv, ctx)
        assert e.value.status == F.FOE_ETIMEOUT
        assert F.foe_server_poll(srv) == []
    finally:
        F.foe_server_destroy(srv)
    assert F.foe_device_status(ctx) == F.FOE_ETIMEOUT
    assert F.foe_device_status(ctx) == F.FOE_OK
    out, _, _ = serve(ctx, ys, [(0, 0), (2, 0)], F.FOE_PREC_BF16, 64 << 20, 4, 5, True)
    refs = reference(ctx, ys, F.FOE_PREC_BF16)
    for j in out:
        assert np.array_equal(out[j], refs[j])
