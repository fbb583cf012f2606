"""The allocation-free resultant entry point (bs_resultant_device_noalloc).

Some callers cannot allocate device memory while they run -- programs whose device
memory belongs to another allocator, latency-critical loops that must not pay for an
allocation.  For them the library offers a resultant whose scratch lives in a static
device array.  This test calls it through the C ABI on device buffers and checks that
calls in a row give exactly what the allocating device entry point gives: two
different curve pairs, then the smaller pair again after the larger one (its leftover
scratch must not leak into the smaller call), in both variables.  It prepares the
context's tables with allocating calls first, so it also passes alone in a fresh
process.
"""

import ctypes as C

import numpy as np
import pytest

pytestmark = pytest.mark.gpu


def _device_grid(torch, bs, f):
    arr, dx, dy, L = bs.bipoly_to_limbs(f)
    t = torch.from_numpy(arr.view(np.int32).copy()).cuda()
    return t, (dx, dy, L)


def test_noalloc_matches_allocating_entry_point():
    torch = pytest.importorskip("torch")
    from paper_1201_1548_gb300.build import build
    build()
    import paper_1201_1548_gb300 as bs
    from paper_1201_1548_gb300._abi import _Bipoly, _Upoly
    from workloads import cfg1_pair, cfg2_pair

    pairs = [cfg1_pair(4), cfg2_pair(5, tdeg=12, bits=32)]
    with bs.Context(0) as ctx:
        lib = ctx.lib
        prepared = {}
        for i, (f, g) in enumerate(pairs):
            tf, mf = _device_grid(torch, bs, f)
            tg, mg = _device_grid(torch, bs, g)
            for var in (1, 0):
                dcap, lcap = ctx.resultant_bounds(mf, mg, var)
                ref = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
                torch.cuda.synchronize()
                # allocating entry point: the reference result (also builds the tables)
                ctx.resultant_device(tf.data_ptr(), mf, tg.data_ptr(), mg, ref.data_ptr(),
                                     (dcap, lcap), var)
                ctx.device_status()
                prepared[i, var] = (tf, mf, tg, mg, dcap, lcap, ref.cpu())
        # allocation-free calls in a row: small, large, small again, then in x
        for key in ((0, 1), (1, 1), (0, 1), (0, 0), (1, 0), (0, 0)):
            tf, mf, tg, mg, dcap, lcap, ref = prepared[key]
            out = torch.full(((dcap + 1) * lcap,), -1, dtype=torch.int32, device="cuda")
            torch.cuda.synchronize()
            fb = _Bipoly(mf[0], mf[1], mf[2], tf.data_ptr())
            gb = _Bipoly(mg[0], mg[1], mg[2], tg.data_ptr())
            ob = _Upoly(dcap, lcap, out.data_ptr())
            rc = lib.bs_resultant_device_noalloc(ctx.h, C.byref(fb), C.byref(gb), key[1],
                                                 C.byref(ob))
            assert rc == 0, lib.bs_last_error_detail(ctx.h).decode()
            ctx.device_status()
            assert torch.equal(out.cpu(), ref), key
            got = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
            assert any(got)
        # a problem whose scratch exceeds the static array is rejected, not computed
        # (an allocating call first prepares the tables, so the size check is the one hit)
        f, g = cfg2_pair(1)
        tf, mf = _device_grid(torch, bs, f)
        tg, mg = _device_grid(torch, bs, g)
        dcap, lcap = ctx.resultant_bounds(mf, mg)
        out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        ctx.resultant_device(tf.data_ptr(), mf, tg.data_ptr(), mg, out.data_ptr(), (dcap, lcap))
        ctx.device_status()
        fb = _Bipoly(mf[0], mf[1], mf[2], tf.data_ptr())
        gb = _Bipoly(mg[0], mg[1], mg[2], tg.data_ptr())
        ob = _Upoly(dcap, lcap, out.data_ptr())
        rc = lib.bs_resultant_device_noalloc(ctx.h, C.byref(fb), C.byref(gb), 1, C.byref(ob))
        assert rc == 7  # BS_ERR_RANGE
        assert "scratch" in lib.bs_last_error_detail(ctx.h).decode()
