"""Bit-exact parity at the full sizes of the workloads, every coefficient.

The expected values were written by ``tests/golden/make_golden.py`` from the oracle alone
(exact Sylvester determinants, Sec. 2, at integer points and exact interpolation); none
comes from the CUDA path.  Where a file stores a SHA-256 digest of a coefficient list
written as comma-separated decimal integers, equal digests mean equal lists.  Results
too large for the oracle (served jobs with degree bound above 800) are checked
coefficient by coefficient modulo the Mersenne prime 2^61 - 1, which is outside the
library's prime table, and exactly at x = 0 and x = 1.

The launch configurations are the ones ``bench.py`` times: the device-planned entry
point on a dedicated stream, the batched graph launch with default and autotuned shapes,
and the serving loop with three slots and batches of at most 16 jobs.
"""

import gzip
import hashlib
import json
import os
import sys

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import poly as P
from workloads import cfg2_pair, cfg3_batch, cfg4_cases, cfg5_stream

pytestmark = pytest.mark.gpu

sys.set_int_max_str_digits(0)
GOLD = os.path.join(os.path.dirname(os.path.abspath(__file__)), "golden")


def _digest(coeffs):
    return hashlib.sha256(",".join(str(int(c)) for c in coeffs).encode()).hexdigest()


def _json(name):
    with open(os.path.join(GOLD, name)) as fh:
        return json.load(fh)


def _cfg2_golden():
    coeffs, deg = [], None
    with gzip.open(os.path.join(GOLD, "cfg2_seed1.txt.gz"), "rt") as fh:
        for line in fh:
            if line.startswith("#"):
                continue
            if line.startswith("deg "):
                deg = int(line.split()[1])
                continue
            coeffs.append(int(line))
    assert deg == len(coeffs) - 1
    return coeffs


def _check_record(rec, got, where):
    """Compare one result with its stored record (exact digest, or residues mod q plus
    exact values at 0 and 1)."""
    if rec["check"] == "exact":
        assert len(got) - 1 == rec["deg"], where
        assert _digest(got) == rec["sha256"], where
        return
    q = rec["modulus"]
    assert len(got) - 1 <= rec["deg_bound"], where
    red = P.mod_p(got, q)
    assert len(red) - 1 == rec["deg_mod"], where
    assert _digest(red) == rec["sha256_mod"], where
    at = rec["at"]
    assert _digest([got[0] if got else 0]) == at["0"], where
    assert _digest([sum(got)]) == at["1"], where


def test_cfg2_every_coefficient_host_buffers(ctx):
    """res(f, f_y; y) of the dense degree-32 curve with 32-bit coefficients: all 993
    coefficients through bs_resultant (host buffers)."""
    f, g = cfg2_pair(1)
    assert ctx.resultant(f, g) == _cfg2_golden()


def test_cfg2_every_coefficient_device_path(ctx):
    """The same resultant through the device-planned entry point on a dedicated stream,
    as bench.py times it, twice in a row (the second call reuses the workspace)."""
    torch = pytest.importorskip("torch")
    want = _cfg2_golden()
    f, g = cfg2_pair(1)
    af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
    stream = torch.cuda.Stream()
    with bs.Context(0) as c2:
        with torch.cuda.stream(stream):
            c2.set_stream(stream.cuda_stream)
            df = torch.from_numpy(af.view(np.int32).copy()).cuda()
            dg = torch.from_numpy(ag.view(np.int32).copy()).cuda()
            dcap, lcap = c2.resultant_bounds((dxf, dyf, Lf), (dxg, dyg, Lg))
            out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
            for _ in range(2):
                out.zero_()
                stream.synchronize()
                c2.resultant_device(df.data_ptr(), (dxf, dyf, Lf), dg.data_ptr(), (dxg, dyg, Lg),
                                    out.data_ptr(), (dcap, lcap))
                c2.device_status()
                vals = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
                while vals and vals[-1] == 0:
                    vals.pop()
                assert vals == want


def test_psc_cfg2_every_coefficient(ctx):
    """All 31 principal subresultant coefficients of the degree-32 curve and f_y
    (Sec. 3.3), every coefficient."""
    gold = _json("psc_cfg2_seed1.json")
    f, g = cfg2_pair(1)
    got = ctx.psc(f, g)
    assert len(got) == len(gold["psc"]) == 31
    for rec in gold["psc"]:
        i = rec["index"]
        assert len(got[i]) - 1 == rec["deg"], i
        assert _digest(got[i]) == rec["sha256"], i


def test_cfg3_batch_sample_every_coefficient(ctx):
    """4096 ragged pairs in one graph launch: the 256 stored pairs compared in full, with
    the default launch shapes and with the shapes the autotuner picks for this batch."""
    gold = _json("cfg3_seed1_subset.json")
    pairs = cfg3_batch(seed=1, count=4096)
    ctx.set_tune()
    got = ctx.resultant_batch(pairs)
    for rec in gold["results"]:
        i = rec["index"]
        _check_record({"check": "exact", **rec}, got[i], i)
    try:
        ctx.autotune_batch(pairs)
        tuned = ctx.resultant_batch(pairs)
    finally:
        ctx.set_tune()
    assert tuned == got


def test_cfg4_degenerate_full_size(ctx):
    """The degenerate inputs at full size (dense degree-12 factors, 16-bit): f1 f2, the
    square factors f1^2 f2 and f1^2 (R = 0), vertical asymptotes, and a leading row
    divisible by the first table prime (that prime is rejected)."""
    gold = _json("cfg4_seed1.json")
    poison = gold["poison_prime"]
    assert poison == bs.bs_prime_table(1)[0]
    cases = cfg4_cases(seed=1, deg=12, bits=16, poison_prime=poison)
    for name in ("4a", "4c", "4d"):
        got = ctx.resultant(*cases[name])
        _check_record(gold["cases"][name], got, name)
        if name == "4d":
            assert ctx.last_stats()["primes_rejected"] >= 1
    for name in ("4b", "4b2"):
        rec = gold["cases"][name]
        assert rec["deg_mod"] == -1 and rec["at"]["0"] == "0"
        assert ctx.resultant(*cases[name]) == []
    fc, _ = cases["4c"]
    rc = ctx.resultant(*cases["4c"])
    for a in (-2, -1, 0, 1, 3):
        assert P.evaluate(rc, a) == 0
    assert len(fc) == 13


@pytest.fixture
def server():
    srv = bs.Context(0)
    yield srv
    srv.serve_stop()
    srv.close()


def _submit(srv, job):
    if job["kind"] == "gcd":
        return srv.submit(bs.JOB_GCD, job["a"], job["b"])
    return srv.submit(bs.JOB_RESULTANT, job["f"], job["g"])


def test_cfg5_served_stream_alone_and_in_the_mix(ctx, server):
    """The whole served stream (256 jobs, total degree 6..64, 16..256-bit coefficients)
    submitted at once to the serving loop (3 slots, batches <= 16): every result equals
    the same job computed alone, and the first 32 equal the oracle's stored values."""
    gold = _json("cfg5_seed1_first32.json")
    stream = cfg5_stream(seed=1)
    server.serve_start(slots=3, max_batch=16)
    tickets = [_submit(server, job) for job in stream]
    served = []
    for t in tickets:
        assert server.wait(t, 300000)
        status, coeffs, _, _ = server.poll(t)
        assert status == 0
        served.append(coeffs)
    st = server.serve_stats()
    assert st["completed"] == len(stream) and st["max_inflight"] >= 2
    for rec in gold["jobs"]:
        i = rec["index"]
        assert stream[i]["kind"] == rec["kind"]
        _check_record(rec, served[i], i)
    for i, job in enumerate(stream):
        alone = (ctx.gcd_z(job["a"], job["b"]) if job["kind"] == "gcd"
                 else ctx.resultant(job["f"], job["g"]))
        assert served[i] == alone, i
    # every gcd job of the stream: the primitive part of the planted factor divides it
    for i, job in enumerate(stream):
        if job["kind"] == "gcd":
            P.exact_div_z(served[i], P.primitive_part(job["planted"]))
