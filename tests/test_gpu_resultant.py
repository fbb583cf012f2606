"""Parity of the full modular resultant (steps (a)-(e)) with the oracle, bit-exact."""

import random

import numpy as np
import pytest

from oracle import numtheory as nt
from oracle import poly as P
from oracle import resultant as R
from workloads import bimul, cfg1_pair, cfg2_pair, cfg3_batch, cfg4_cases, d_dy, dense_curve

pytestmark = pytest.mark.gpu


def _rng(seed):
    return np.random.Generator(np.random.PCG64(seed))


@pytest.mark.parametrize("seed", [1, 2, 3])
@pytest.mark.parametrize("var", [1, 0])
def test_cfg1_exact(ctx, seed, var):
    f, g = cfg1_pair(seed)
    assert ctx.resultant(f, g, var) == R.resultant(f, g, var)


def test_small_random_pairs_both_variables(ctx):
    rng = _rng(11)
    for t in range(40):
        f = dense_curve(rng, int(rng.integers(1, 7)), int(rng.integers(2, 90)),
                        zero_prob=0.2 if t % 2 else 0.0, keep_top=t % 3 != 0)
        g = dense_curve(rng, int(rng.integers(1, 7)), int(rng.integers(2, 90)),
                        zero_prob=0.2 if t % 2 else 0.0, keep_top=t % 3 != 1)
        for var in (1, 0):
            assert ctx.resultant(f, g, var) == R.resultant(f, g, var), (t, var)


def test_trivial_and_constant_cases(ctx):
    zero = [[0, 0], [0, 0]]
    g = [[1, 2], [3, 0]]
    assert ctx.resultant(zero, g) == []
    assert ctx.resultant(g, zero) == []
    assert ctx.resultant([[5]], [[7, 1]]) == [1]                 # both constant in y
    f0 = [[2, -3, 1]]                                              # f = f_0(x), m_y = 0
    h = [[1, 1], [0, 2], [5, 0]]
    assert ctx.resultant(f0, h) == R.res_y(f0, h)                  # f_0^{n_y}
    assert ctx.resultant(h, f0) == R.res_y(h, f0)
    # high-degree x with y-degree 1 (degree bound from n_y deg_x f + m_y deg_x g)
    f = [[1] + [0] * 40 + [3], [0] * 41 + [0, ]]
    f[1][0] = 1
    gg = [[2, 1], [1, 0]]
    assert ctx.resultant(f, gg) == R.res_y(f, gg)


def test_wide_coefficients_and_high_bits(ctx):
    rng = _rng(12)
    from workloads import highbit_variant
    f = highbit_variant(dense_curve(rng, 4, 20), 512)
    g = d_dy(f)
    assert ctx.resultant(f, g) == R.res_y(f, g)
    f = dense_curve(rng, 3, 1500)
    g = dense_curve(rng, 3, 700)
    assert ctx.resultant(f, g) == R.res_y(f, g)


def test_cfg2_sampled_points(ctx):
    """Discriminant-type resultant of a degree-32 curve with 32-bit coefficients: the
    oracle evaluates R exactly at sampled integer points and mod p at sampled points."""
    f, g = cfg2_pair(1)
    r = ctx.resultant(f, g)
    assert 0 <= P.deg(r) <= R.degree_bound(f, g) == 992
    b2 = R.bound_sq(f, g)
    assert all(c * c <= b2 for c in r)
    for x0 in (0, 1, -1, 3):
        assert P.evaluate(r, x0) == R.res_at_point(f, g, x0), x0
    rng = random.Random(3)
    # primes outside the library's table (2^31 - 1 is not 1 mod 2^14), so a wrong
    # reconstruction cannot agree with them by construction
    for p in (2147483647, (1 << 61) - 1):
        assert p not in nt.prime_table(200)
        for _ in range(3):
            a = rng.randrange(p)
            assert P.evaluate(r, a) % p == R.res_at_point_modp(f, g, a, p)


def test_device_path_matches_host_path(ctx):
    torch = pytest.importorskip("torch")
    import paper_1201_1548_gb300 as bs
    for f, g in [cfg1_pair(1), cfg2_pair(2)] + cfg3_batch(seed=9, count=3):
        host = ctx.resultant(f, g)
        af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
        df = torch.from_numpy(af.view(np.int32).copy()).cuda()
        dg = torch.from_numpy(ag.view(np.int32).copy()).cuda()
        dcap, lcap = ctx.resultant_bounds((dxf, dyf, Lf), (dxg, dyg, Lg))
        out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
        torch.cuda.synchronize()
        ctx.resultant_device(df.data_ptr(), (dxf, dyf, Lf), dg.data_ptr(), (dxg, dyg, Lg),
                             out.data_ptr(), (dcap, lcap))
        ctx.device_status()
        vals = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
        while vals and vals[-1] == 0:
            vals.pop()
        assert vals == host


def _device_call(ctx, f, g):
    torch = pytest.importorskip("torch")
    import paper_1201_1548_gb300 as bs
    af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
    df = torch.from_numpy(af.view(np.int32).copy()).cuda()
    dg = torch.from_numpy(ag.view(np.int32).copy()).cuda()
    dcap, lcap = ctx.resultant_bounds((dxf, dyf, Lf), (dxg, dyg, Lg))
    out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    ctx.resultant_device(df.data_ptr(), (dxf, dyf, Lf), dg.data_ptr(), (dxg, dyg, Lg),
                         out.data_ptr(), (dcap, lcap))
    ctx.device_status()
    vals = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
    while vals and vals[-1] == 0:
        vals.pop()
    return vals


def test_device_path_large_transforms(ctx):
    """Device-planned jobs with 2048- and 4096-point sets (the plan is made on the device, so
    the size-class dispatch and the shared-memory transform run from device-side offsets)
    give what the host path gives; the last pair has rows of 1101 coefficients, folded
    modulo N."""
    import paper_1201_1548_gb300 as bs
    rng = _rng(77)
    pairs = []
    for tdeg, bits in ((40, 8), (48, 6)):
        f = dense_curve(rng, tdeg, bits)
        pairs.append((f, d_dy(f)))
    f = [[int(v) for v in rng.integers(-99, 100, 1101)] for _ in range(3)]  # deg_y 2, deg_x 1100
    pairs.append((f, d_dy(f)))
    for f, g in pairs:
        assert bs.bs_plan(f, g)["N"] >= 2048
        dev = _device_call(ctx, f, g)
        assert dev == ctx.resultant(f, g)
        p = 2147483647  # outside the library's table
        for x0 in (3, 12345):
            assert P.evaluate(dev, x0) % p == R.res_at_point_modp(f, g, x0, p)


def test_large_transform_rows_of_65_to_96_coefficients(ctx):
    """Rows of 81 coefficients at 2048 points: the stages of the shared-memory transform
    that combine points 1024 apart leave only the first three registers of each warp's
    chunk nonzero, and the warp runs its pruned 1024-point variant.  The host and device
    paths give the oracle's resultant coefficient by coefficient."""
    import paper_1201_1548_gb300 as bs
    rng = _rng(88)
    f = [[int(v) for v in rng.integers(-99, 100, 81)] for _ in range(8)]  # deg_y 7, deg_x 80
    g = d_dy(f)
    assert bs.bs_plan(f, g)["N"] == 2048
    want = R.res_y(f, g)
    assert len(want) == 1041
    assert ctx.resultant(f, g) == want
    assert _device_call(ctx, f, g) == want


def test_device_plan_exact_spares(ctx):
    """Single-coefficient leading rows: the device plan counts exactly the table primes that
    divide them.  With lc_y f = p_0 p_1 (two table primes) those two are rejected and
    replaced; with lc_y f = 1 no spare is evaluated.  Both results equal the oracle's."""
    import paper_1201_1548_gb300 as bs
    rng = _rng(41)
    p0, p1 = nt.prime_table(2)
    for lc in (p0 * p1, 1):
        f = dense_curve(rng, 9, 12)
        f[-1] = [lc] + [0] * (len(f[-1]) - 1)   # leading row in y: the constant lc
        g = d_dy(f)
        before = bs.bs_plan(f, g)
        dev = _device_call(ctx, f, g)
        assert dev == R.res_y(f, g)
        assert before["k_total"] == before["k_need"] + (2 if lc != 1 else 0)


def test_degenerate_cfg4(ctx):
    cases = cfg4_cases(seed=1, deg=5, bits=12, poison_prime=nt.prime_table(1)[0])
    # square factors: res_y(f, f_y) vanishes identically
    assert ctx.resultant(*cases["4b"]) == []
    assert ctx.resultant(*cases["4b2"]) == []
    # f = f1 f2: exact against the oracle
    fa, ga = cases["4a"]
    assert ctx.resultant(fa, ga) == R.res_y(fa, ga)
    # vertical asymptotes at x in {-2, -1, 0, 1, 3}: both leading coefficients vanish
    fc, gc = cases["4c"]
    rc = ctx.resultant(fc, gc)
    assert rc == R.res_y(fc, gc)
    for a in (-2, -1, 0, 1, 3):
        assert P.evaluate(rc, a) == 0
    # a table prime divides lc_y f: that prime is rejected, the result stays exact
    fd, gd = cases["4d"]
    assert ctx.resultant(fd, gd) == R.res_y(fd, gd)
    assert ctx.last_stats()["primes_rejected"] >= 1


def test_point_rejection_on_coset(ctx):
    """lc_y f has a root at a point of the first prime's evaluation set: that prime is
    rejected and the result is still exact."""
    f0, g0 = cfg1_pair(5)
    plan_n = 64                       # N for total degrees 7 x 6 (D <= 42)
    p = nt.prime_table(1)[0]
    pts = nt.coset_points(p, plan_n)
    a = pts[5]
    # f = (x - a) y^6 + (random lower rows)
    f = [row + [0] for row in f0]
    f[6] = [-a, 1] + [0] * (len(f[0]) - 2)
    g = d_dy(f)
    import paper_1201_1548_gb300 as bs
    assert bs.bs_plan(f, g)["N"] == plan_n
    r = ctx.resultant(f, g)
    assert r == R.res_y(f, g)
    assert ctx.last_stats()["primes_rejected"] >= 1


def test_unlucky_job_fails_cleanly_and_context_stays_usable(ctx):
    """A leading coefficient vanishing at a point of the first three primes' evaluation
    sets (their coset representatives are roots of lc_y f) rejects three primes, one more
    than the host plan's two spares: the call reports BS_ERR_UNLUCKY (the reconstruction
    reads no unset selection slot), and so does the device-planned entry point unless its
    own spare count covers them (then its result is exact); later calls on the context
    are exact."""
    import paper_1201_1548_gb300 as bs
    torch = pytest.importorskip("torch")
    rng = _rng(31)
    f = dense_curve(rng, 5, 12)
    lc = [1]
    for p in nt.prime_table(3):
        lc = P.mul(lc, [-nt.coset_representative(p), 1])    # (x - c_0)(x - c_1)(x - c_2)
    width = max(len(lc), len(f[0]))
    f = [row + [0] * (width - len(row)) for row in f]
    f[5] = lc + [0] * (width - len(lc))
    g = d_dy(f)
    plan = bs.bs_plan(f, g)
    assert plan["k_total"] - plan["k_need"] == 2
    with pytest.raises(bs.BsError) as e:
        ctx.resultant(f, g)
    assert e.value.code == bs.BS_ERR_UNLUCKY
    af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
    df = torch.from_numpy(af.view(np.int32).copy()).cuda()
    dg = torch.from_numpy(ag.view(np.int32).copy()).cuda()
    dcap, lcap = ctx.resultant_bounds((dxf, dyf, Lf), (dxg, dyg, Lg))
    out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
    torch.cuda.synchronize()
    ctx.resultant_device(df.data_ptr(), (dxf, dyf, Lf), dg.data_ptr(), (dxg, dyg, Lg),
                         out.data_ptr(), (dcap, lcap))
    try:
        ctx.device_status()
    except bs.BsError as e:
        assert e.code == bs.BS_ERR_UNLUCKY
    else:
        vals = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
        while vals and vals[-1] == 0:
            vals.pop()
        assert vals == R.res_y(f, g)
    f1, g1 = cfg1_pair(2)
    assert ctx.resultant(f1, g1) == R.res_y(f1, g1)


def test_batch_matches_single_and_oracle(ctx):
    pairs = cfg3_batch(seed=21, count=48, deg_lo=2, deg_hi=7, bits_lo=8, bits_hi=64)
    got = ctx.resultant_batch(pairs)
    for (f, g), r in zip(pairs, got):
        assert r == R.res_y(f, g)
        assert r == ctx.resultant(f, g)


@pytest.mark.parametrize("tdeg,bits", [(40, 8), (48, 6)])
def test_large_transforms_sampled(ctx, tdeg, bits):
    """D >= 1024 (2048- and 4096-point sets: the shared-memory transform path)."""
    rng = _rng(100 + tdeg)
    f = dense_curve(rng, tdeg, bits)
    g = d_dy(f)
    import paper_1201_1548_gb300 as bs
    assert bs.bs_plan(f, g)["N"] >= 2048
    r = ctx.resultant(f, g)
    assert P.deg(r) <= R.degree_bound(f, g)
    for x0 in (0, 1, -2):
        assert P.evaluate(r, x0) == R.res_at_point(f, g, x0)
    p = 2147483647  # outside the library's table
    assert P.evaluate(r, 12345) % p == R.res_at_point_modp(f, g, 12345, p)


def test_cfg3_full_batch_sampled(ctx):
    """4096 pairs of uneven degree (4-24) and coefficient size (8-64 bits) in one graph
    launch: exact oracle results for the small pairs, exact values at integer points and
    values mod a prime outside the working set for a seeded sample of the rest."""
    pairs = cfg3_batch(seed=1, count=4096)
    got = ctx.resultant_batch(pairs)
    assert len(got) == len(pairs)
    rng = random.Random(5)
    p = 2147483647  # a prime outside the library's table (2^31 - 1 is not 1 mod 2^14)
    assert nt.is_prime(p)
    for i in rng.sample(range(len(pairs)), 48):
        f, g = pairs[i]
        r = got[i]
        assert P.deg(r) <= R.degree_bound(f, g)
        a = rng.randrange(p)
        assert P.evaluate(r, a) % p == R.res_at_point_modp(f, g, a, p), i
    for i in rng.sample(range(len(pairs)), 8):
        f, g = pairs[i]
        assert P.evaluate(got[i], 1) == R.res_at_point(f, g, 1), i
        assert got[i] == ctx.resultant(f, g), i
    small = [i for i in range(len(pairs)) if len(pairs[i][0]) + len(pairs[i][1]) <= 12][:12]
    for i in small:
        assert got[i] == R.res_y(*pairs[i]), i


@pytest.mark.parametrize("tdeg,bits", [(8, 600), (16, 256)])
def test_many_primes_block_reconstruction(ctx, tdeg, bits):
    """k above the warp reconstruction's limit (the block Garner path): exact values at
    integer points and values mod a prime outside the table."""
    import paper_1201_1548_gb300 as bs
    rng = _rng(200 + tdeg)
    f = dense_curve(rng, tdeg, bits)
    g = dense_curve(rng, tdeg, bits)
    info = bs.bs_plan(f, g)
    assert info["k_need"] > 160
    r = ctx.resultant(f, g)
    assert P.deg(r) <= R.degree_bound(f, g)
    b2 = R.bound_sq(f, g)
    assert all(c * c <= b2 for c in r)
    for x0 in (0, 1, -1):
        assert P.evaluate(r, x0) == R.res_at_point(f, g, x0)
    p = 2147483647
    for a in (12345, 987654321):
        assert P.evaluate(r, a) % p == R.res_at_point_modp(f, g, a, p)


def test_largest_served_size(ctx):
    """The largest job of the served stream (total degree 64, 256-bit coefficients:
    about 1150 primes and 8192 points per prime): values mod a prime outside the table."""
    import paper_1201_1548_gb300 as bs
    rng = _rng(300)
    f = dense_curve(rng, 64, 256)
    g = dense_curve(rng, 64, 256)
    info = bs.bs_plan(f, g)
    assert info["N"] == 8192 and info["k_need"] > 1000
    r = ctx.resultant(f, g)
    assert P.deg(r) <= R.degree_bound(f, g)
    p = 2147483647
    for a in (3, 1234567):
        assert P.evaluate(r, a) % p == R.res_at_point_modp(f, g, a, p)


@pytest.mark.parametrize("shape", [
    dict(eval_warps=2, eval_blocks_per_sm=4, uni_threads=(64,) * 6, crt_tile=2, crt_blocks_per_sm=2,
         eval_independent=0),
    dict(eval_warps=4, eval_blocks_per_sm=16, uni_threads=(256,) * 6, crt_tile=4, crt_blocks_per_sm=8,
         eval_independent=0),
    dict(eval_warps=1, eval_blocks_per_sm=1, uni_threads=(64, 128, 256, 64, 128, 256), crt_tile=1,
         crt_blocks_per_sm=1),
])
def test_batch_results_do_not_depend_on_launch_shape(ctx, shape):
    pairs = cfg3_batch(seed=23, count=64, deg_lo=2, deg_hi=12, bits_lo=8, bits_hi=96)
    ctx.set_tune()
    ref = ctx.resultant_batch(pairs)
    ctx.set_tune(**shape)
    try:
        assert ctx.resultant_batch(pairs) == ref
        assert ctx.resultant(*pairs[5]) == ref[5]
    finally:
        ctx.set_tune()
    for i in range(0, 64, 16):
        assert ref[i] == R.res_y(*pairs[i])


def test_autotune_batch(ctx):
    pairs = cfg3_batch(seed=24, count=256)
    ref = ctx.resultant_batch(pairs)
    info = ctx.autotune_batch(pairs)
    try:
        assert info["trials"] >= 3
        assert info["eval_warps"] in (2, 4, 8) and info["crt_tile"] in (2, 4, 8)
        assert info["eval_independent"] in (0, 1)
        assert all(t in (64, 128, 256) for t in info["uni_threads"])
        assert 0 < info["ms_tuned"] <= 1.1 * info["ms_default"]
        assert ctx.resultant_batch(pairs) == ref
    finally:
        ctx.set_tune()


def test_many_primes_with_a_rejected_prime(ctx):
    """k above the warp limit and the first table prime dividing the leading row: that
    prime is rejected, so the selection is not the first k table primes and the block
    Garner kernel reconstructs this job."""
    import paper_1201_1548_gb300 as bs
    p0 = bs.bs_prime_table(1)[0]
    rng = _rng(210)
    f = dense_curve(rng, 8, 600)
    f[8] = [c * p0 for c in f[8]]
    g = d_dy(f)
    assert bs.bs_plan(f, g)["k_need"] > 160
    r = ctx.resultant(f, g)
    assert ctx.last_stats()["primes_rejected"] >= 1
    for x0 in (0, 1, -1):
        assert P.evaluate(r, x0) == R.res_at_point(f, g, x0)
    p = 2147483647
    assert P.evaluate(r, 4242) % p == R.res_at_point_modp(f, g, 4242, p)
    # the same job inside a batch next to jobs with few and with many primes
    small = cfg1_pair(2)
    big = (dense_curve(rng, 8, 600), dense_curve(rng, 8, 600))
    got = ctx.resultant_batch([small, (f, g), big])
    assert got[0] == R.res_y(*small)
    assert got[1] == r
    assert got[2] == ctx.resultant(*big)
