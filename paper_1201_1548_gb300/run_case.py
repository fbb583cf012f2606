"""Run one of the benchmark workloads a given number of times (for profilers).

    python -m paper_1201_1548_gb300.run_case discriminant32 [reps]
        res_y(f, df/dy) of a dense curve of total degree 32 with 32-bit coefficients,
        device-resident inputs (bs_resultant_device), one call per repetition.
    python -m paper_1201_1548_gb300.run_case batch4096 [reps]
        4096 pairs of total degrees 4..24 and 8..64-bit coefficients through
        bs_resultant_batch (one graph launch per repetition).
    python -m paper_1201_1548_gb300.run_case projection32 [reps]
        the square-free part, Yun's factorisation and the psc sequence of the degree-32
        curve's resultant R = res(f, f_y) (deg 992), one call each per repetition.

Each run checks its result against the host entry point once and prints "ok".
"""

from __future__ import annotations

import os
import sys


def _discriminant32(reps):
    import numpy as np
    import torch

    import paper_1201_1548_gb300 as bs
    from workloads import cfg2_pair

    f, g = cfg2_pair(1)
    ctx = bs.Context(0)
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream.cuda_stream)
    af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
    df = torch.from_numpy(af.view(np.int32).copy()).cuda()
    dg = torch.from_numpy(ag.view(np.int32).copy()).cuda()
    dcap, lcap = ctx.resultant_bounds((dxf, dyf, Lf), (dxg, dyg, Lg))
    out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    for _ in range(reps):
        ctx.resultant_device(df.data_ptr(), (dxf, dyf, Lf), dg.data_ptr(), (dxg, dyg, Lg),
                             out.data_ptr(), (dcap, lcap))
        ctx.device_status()
    dev = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
    while dev and dev[-1] == 0:
        dev.pop()
    if dev != ctx.resultant(f, g):
        raise SystemExit("device and host results differ")


def _batch4096(reps):
    import paper_1201_1548_gb300 as bs
    from workloads import cfg3_batch

    pairs = cfg3_batch(seed=1, count=4096)
    ctx = bs.Context(0)
    first = None
    for _ in range(reps):
        got = ctx.resultant_batch(pairs)
        first = first or got
    for i in range(0, len(pairs), 512):
        if first[i] != ctx.resultant(*pairs[i]):
            raise SystemExit(f"batched and single results differ at pair {i}")


def _projection32(reps):
    import time

    import paper_1201_1548_gb300 as bs
    from workloads import cfg2_pair

    f, g = cfg2_pair(1)
    ctx = bs.Context(0)
    R = ctx.resultant(f, g)
    for _ in range(reps):
        t0 = time.perf_counter()
        sq = ctx.squarefree_part(R)
        t1 = time.perf_counter()
        fac = ctx.squarefree_factorization(R)
        t2 = time.perf_counter()
        ps = ctx.psc(f, g)
        t3 = time.perf_counter()
        print(f"sqf {1e3 * (t1 - t0):.2f} ms  yun {1e3 * (t2 - t1):.2f} ms  psc {1e3 * (t3 - t2):.2f} ms")
    if fac[-1] != sq and len(fac) == 1 or ps[0] != R:
        raise SystemExit("inconsistent projection results")


CASES = {"discriminant32": _discriminant32, "batch4096": _batch4096, "projection32": _projection32}


def main(argv):
    root = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
    if root not in sys.path:
        sys.path.insert(0, root)
    if not argv or argv[0] not in CASES:
        raise SystemExit(f"usage: python -m paper_1201_1548_gb300.run_case {{{'|'.join(CASES)}}} [reps]")
    reps = int(argv[1]) if len(argv) > 1 else 2
    CASES[argv[0]](reps)
    print("ok")


if __name__ == "__main__":
    main(sys.argv[1:])
