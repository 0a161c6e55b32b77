"""The tensor-core cost probe (foe_mma_cost) on the device: every one-CTA shape of the table runs, and the shapes
order as the shared-memory operand model says: per multiply-add, a wide N costs fewer cycles than the N = 64 / 96
of the step kernels, and no shape exceeds the tensor pipe's dense rate (4096 multiply-adds per clock and SM)."""
import pytest

torch = pytest.importorskip("torch")

from paper_1609_05722_gb300 import build as B  # noqa: E402
from paper_1609_05722_gb300 import foe as F  # noqa: E402
from paper_1609_05722_gb300 import mma_cost as M  # noqa: E402

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def built():
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    B.build()
    torch.cuda.set_device(0)


def test_every_single_cta_shape_runs():
    rows = [M.row(m, n, a, False, iss, 512) for m, n, a, iss in M.SINGLE]
    for r in rows:
        assert 0.0 < r["mac_per_clk_sm"] <= 4096 * 1.05, r


def test_wide_n_costs_fewer_cycles_per_mac():
    n64 = M.row(128, 64, False, False, 2, 1024)
    n256 = M.row(128, 256, False, False, 2, 1024)
    assert n256["mac_per_clk_sm"] > 1.5 * n64["mac_per_clk_sm"], (n64, n256)


def test_sm_pair_shapes_run():
    # cta_group::2: M = 256 over the two SMs of a cluster, each reading half of B
    for m, n, a, iss in M.PAIR:
        r = M.row(m, n, a, True, iss, 512)
        assert 0.0 < r["mac_per_clk_sm"] <= 4096 * 1.05, r
