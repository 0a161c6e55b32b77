"""Tensor-core contraction ceilings by MMA shape and operand source (``foe_mma_cost``), printed as a table.

    python -m paper_1609_05722_gb300.mma_cost            # one-CTA shapes (cta_group::1)
    python -m paper_1609_05722_gb300.mma_cost --pair     # M = 256 over an SM pair (cta_group::2)

Each row gives the SM cycles per tcgen05.mma (kind::f16, K = 16), the multiply-adds per clock and SM that this
implies, its share of 4096 (the dense BF16 rate of an SM's tensor pipe: 128 x 256 x 16 multiply-adds in 128 clocks),
and the shared-memory operand bytes each SM reads per clock.  The step kernels' forward responses are M = 128 pixel
pairs x N = 96 (two pixels x 48 filters, Eq. FoEF) with A from shared memory, their adjoint M = 128 x N = 64 with A
(the expert derivative) from tensor memory.
"""
from __future__ import annotations

import argparse
import json

from . import foe as F

# (m, n, A in tensor memory, issuing warps)
SINGLE = [
    (128, 48, False, 2), (128, 64, False, 2), (128, 96, False, 2), (128, 128, False, 2), (128, 256, False, 2),
    (128, 256, False, 1), (64, 64, False, 2), (64, 256, False, 2),
    (128, 64, True, 2), (128, 96, True, 2), (128, 128, True, 2), (128, 256, True, 1),
]
PAIR = [(256, 64, False, 2), (256, 96, False, 2), (256, 128, False, 2), (256, 256, False, 2)]


def row(m: int, n: int, a_tmem: bool, pair: bool, issuers: int, count: int) -> dict:
    cyc = F.foe_mma_cost(m, n, a_tmem, pair, issuers, count)
    rows_per_sm = m // 2 if pair else m
    macs = rows_per_sm * n * 16
    # operand bytes read from this SM's shared memory per MMA: its rows of A (unless in tensor memory) and of B
    smem_bytes = (0 if a_tmem else rows_per_sm * 32) + (n // 2 if pair else n) * 32
    return {"m": m, "n": n, "a": "tmem" if a_tmem else "smem", "cta_group": 2 if pair else 1, "issuers": issuers,
            "cycles_per_mma": round(cyc, 2), "mac_per_clk_sm": round(macs / cyc, 1),
            "of_4096": round(macs / cyc / 4096.0, 3), "smem_bytes_per_clk": round(smem_bytes / cyc, 1)}


def main(argv=None) -> None:
    ap = argparse.ArgumentParser(description=__doc__.splitlines()[0])
    ap.add_argument("--pair", action="store_true", help="the cta_group::2 shapes instead of the one-CTA shapes")
    ap.add_argument("--count", type=int, default=4096, help="MMAs per issuing warp")
    ap.add_argument("--json", action="store_true", help="one JSON object per row")
    args = ap.parse_args(argv)
    cases = PAIR if args.pair else SINGLE
    hdr = "   m    n  A     group issuers  clk/MMA  MAC/clk/SM  of 4096  smem B/clk"
    if not args.json:
        print(hdr)
    for m, n, a_tmem, iss in cases:
        r = row(m, n, a_tmem, args.pair, iss, args.count)
        if args.json:
            print(json.dumps(r))
        else:
            print(f"{m:4d} {n:4d}  {r['a']:5s} {r['cta_group']:5d} {iss:7d} {r['cycles_per_mma']:8.1f} "
                  f"{r['mac_per_clk_sm']:11.1f} {r['of_4096']:8.3f} {r['smem_bytes_per_clk']:11.1f}", flush=True)


if __name__ == "__main__":
    main()
