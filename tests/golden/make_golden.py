"""Writes the stored expected values of the full-size parity tests (test infrastructure).

Every stored value is computed here by the oracle (``oracle/``) from the seeded inputs of
``workloads/``; this script imports nothing else of the repository and never touches the
CUDA path.  The files it writes next to itself:

* ``cfg2_seed1.txt.gz`` -- every coefficient of R = res(f, f_y; y) for the dense curve
  of total degree 32 with signed 32-bit coefficients (``cfg2_pair(1)``), one decimal
  integer per line (R = det of the Sylvester matrix of Sec. 2; points route of the
  oracle: exact Bareiss determinants at D + 1 = 993 integer points and exact Newton
  interpolation).
* ``cfg3_seed1_subset.json`` -- a seeded sample of 256 of the 4096 ragged pairs of
  ``cfg3_batch(seed=1)``: the degree of each exact resultant and the SHA-256 digest of
  its coefficients written as comma-separated decimal integers (equal digests mean
  equal coefficient lists).
* ``cfg4_seed1.json`` -- the degenerate inputs at full size (two dense degree-12 curves
  with 16-bit coefficients): exact results of 4a, 4c and 4d; 4b and 4b2 (square factors,
  R = 0) modulo a prime outside the library's table and exactly at x = 0.
* ``cfg5_seed1_first32.json`` -- the first 32 jobs of the served stream
  ``cfg5_stream(seed=1)``: gcd jobs exactly (the oracle's gcd in Z[x]); resultant jobs
  exactly where the oracle finishes in minutes (degree bound <= 800), otherwise every
  coefficient modulo the Mersenne prime 2^61 - 1 (outside the library's prime table)
  together with the exact values R(0) and R(1).

* ``psc_cfg2_seed1.json`` -- the 31 principal subresultant coefficients sr_0 ... sr_30 of
  the same f and f_y with respect to y (Sec. 3.3), each as degree and digest.

Usage: ``python tests/golden/make_golden.py [--procs N] [--only cfg2,cfg3,cfg4,cfg5,psc2]``.
The point determinants run on a spawned process pool; the wall time per file and the
process count are written into each file.
"""

from __future__ import annotations

import argparse
import gzip
import hashlib
import json
import multiprocessing as mp
import os
import random
import sys
import time

HERE = os.path.dirname(os.path.abspath(__file__))
ROOT = os.path.dirname(os.path.dirname(HERE))
if ROOT not in sys.path:
    sys.path.insert(0, ROOT)

sys.set_int_max_str_digits(0)  # exact values of tens of thousands of digits

from oracle import gcd as G  # noqa: E402
from oracle import resultant as R  # noqa: E402
from oracle import subresultant as S  # noqa: E402
from oracle.numtheory import prime_table  # noqa: E402
from workloads import cfg2_pair, cfg3_batch, cfg4_cases, cfg5_stream  # noqa: E402

Q61 = (1 << 61) - 1          # modulus of the reduced checks (not in the library's table)
CFG3_SAMPLE = 256            # pairs of the 4096-pair batch with stored digests
CFG3_SAMPLE_SEED = 1         # random.Random seed of that sample
CFG5_JOBS = 32               # leading jobs of the served stream
CFG5_EXACT_MAX_D = 800       # resultant jobs up to this degree bound are stored exactly


def digest(coeffs):
    """SHA-256 of the coefficient list written as comma-separated decimal integers."""
    return hashlib.sha256(",".join(str(int(c)) for c in coeffs).encode()).hexdigest()


def cfg3_sample_indices(count=4096):
    return sorted(random.Random(CFG3_SAMPLE_SEED).sample(range(count), CFG3_SAMPLE))


# ---- pool tasks (module level so that a spawned worker can import them) ----------------

def _whole_resultant(args):
    f, g = args
    return R.res_y(f, g)


def _gcd_task(args):
    a, b = args
    return G.gcd_z(a, b)


def _point_task(args):
    f, g, x0 = args
    return R.res_at_point(f, g, x0)


def _write_json(name, obj):
    path = os.path.join(HERE, name)
    with open(path, "w") as fh:
        json.dump(obj, fh, indent=1)
        fh.write("\n")
    print(f"wrote {path}", flush=True)


def make_cfg2(pool, procs):
    f, g = cfg2_pair(1)
    t0 = time.time()
    r = R.res_y(f, g, map=lambda fn, xs: pool.map(fn, xs, chunksize=4))
    dt = time.time() - t0
    path = os.path.join(HERE, "cfg2_seed1.txt.gz")
    with gzip.open(path, "wt") as fh:
        fh.write("# R = res(f, f_y; y), f = workloads.cfg2_pair(1)[0]: dense, total degree 32,\n")
        fh.write("# signed 32-bit coefficients.  Written by tests/golden/make_golden.py from the\n")
        fh.write("# oracle's points route (Sec. 2 Sylvester determinant at 993 integer points,\n")
        fh.write("# exact Newton interpolation).\n")
        fh.write(f"# oracle wall time {dt:.1f} s on {procs} processes\n")
        fh.write(f"deg {len(r) - 1}\n")
        for c in r:
            fh.write(f"{c}\n")
    print(f"wrote {path}: deg {len(r) - 1}, {dt:.1f} s", flush=True)
    return dt


def make_cfg3(pool, procs):
    pairs = cfg3_batch(seed=1, count=4096)
    idx = cfg3_sample_indices(len(pairs))
    # longest first, so the pool's tail stays short
    order = sorted(idx, key=lambda i: -(R.degree_bound(*pairs[i]) + 1)
                   * (len(pairs[i][0]) + len(pairs[i][1])) ** 3)
    t0 = time.time()
    res = dict(zip(order, pool.map(_whole_resultant, [pairs[i] for i in order], chunksize=1)))
    dt = time.time() - t0
    out = {
        "recipe": "workloads.cfg3_batch(seed=1, count=4096); sample = sorted(random.Random(1)"
                  ".sample(range(4096), 256)); res(f, g; y) by oracle.resultant.res_y",
        "digest": "sha256 of the coefficients (ascending) as comma-separated decimal integers",
        "oracle_seconds": round(dt, 1), "processes": procs,
        "results": [{"index": i, "deg": len(res[i]) - 1, "sha256": digest(res[i])} for i in idx],
    }
    _write_json("cfg3_seed1_subset.json", out)
    return dt


def make_cfg4(pool, procs):
    poison = prime_table(1)[0]
    cases = cfg4_cases(seed=1, deg=12, bits=16, poison_prime=poison)
    t0 = time.time()
    out = {"recipe": f"workloads.cfg4_cases(seed=1, deg=12, bits=16, poison_prime={poison})"
                     " (the first prime of the table); g = df/dy",
           "digest": "sha256 of the coefficients (ascending) as comma-separated decimal integers",
           "modulus": Q61, "poison_prime": poison, "cases": {}}
    for name in ("4a", "4c", "4d"):
        f, g = cases[name]
        r = R.res_y(f, g, map=lambda fn, xs: pool.map(fn, xs, chunksize=2))
        out["cases"][name] = {"check": "exact", "deg": len(r) - 1, "sha256": digest(r)}
        print(f"cfg4 {name}: deg {len(r) - 1}", flush=True)
    for name in ("4b", "4b2"):
        f, g = cases[name]
        rq = R.res_y_modp(f, g, Q61, map=lambda fn, xs: pool.map(fn, xs, chunksize=8))
        v0 = R.res_at_point(f, g, 0)
        out["cases"][name] = {"check": "mod", "deg_bound": R.degree_bound(f, g),
                              "deg_mod": len(rq) - 1, "sha256_mod": digest(rq),
                              "at": {"0": str(v0)}}
        print(f"cfg4 {name}: deg mod q {len(rq) - 1}, R(0) = {v0}", flush=True)
    dt = time.time() - t0
    out["oracle_seconds"] = round(dt, 1)
    out["processes"] = procs
    _write_json("cfg4_seed1.json", out)
    return dt


def make_psc_cfg2(pool, procs):
    f, g = cfg2_pair(1)
    t0 = time.time()
    sr = S.psc_y(f, g, map=lambda fn, xs: pool.map(fn, xs, chunksize=4))
    dt = time.time() - t0
    out = {"recipe": "workloads.cfg2_pair(1); [sr_0, ..., sr_30] of f and f_y with respect to y "
                     "by oracle.subresultant.psc_y (points route)",
           "digest": "sha256 of the coefficients (ascending) as comma-separated decimal integers",
           "oracle_seconds": round(dt, 1), "processes": procs,
           "psc": [{"index": i, "deg": len(s) - 1, "sha256": digest(s)} for i, s in enumerate(sr)]}
    _write_json("psc_cfg2_seed1.json", out)
    return dt


def make_cfg5(pool, procs):
    stream = cfg5_stream(seed=1)[:CFG5_JOBS]
    t0 = time.time()
    recs = [None] * len(stream)
    # whole-job tasks: gcds and the exact resultants of small degree bound
    small = []
    for i, job in enumerate(stream):
        if job["kind"] == "gcd":
            small.append((i, _gcd_task, (job["a"], job["b"])))
    gres = pool.map(_gcd_task, [a for (_, _, a) in small], chunksize=1)
    for (i, _, _), h in zip(small, gres):
        recs[i] = {"index": i, "kind": "gcd", "check": "exact", "deg": len(h) - 1,
                   "sha256": digest(h)}
    for i, job in enumerate(stream):
        if job["kind"] != "resultant":
            continue
        f, g = job["f"], job["g"]
        D = R.degree_bound(f, g)
        if D <= CFG5_EXACT_MAX_D:
            r = R.res_y(f, g, map=lambda fn, xs: pool.map(fn, xs, chunksize=1))
            recs[i] = {"index": i, "kind": "resultant", "check": "exact", "deg": len(r) - 1,
                       "sha256": digest(r)}
        else:
            rq = R.res_y_modp(f, g, Q61, map=lambda fn, xs: pool.map(fn, xs, chunksize=8))
            v = pool.map(_point_task, [(f, g, 0), (f, g, 1)], chunksize=1)
            recs[i] = {"index": i, "kind": "resultant", "check": "mod", "deg_bound": D,
                       "modulus": Q61, "deg_mod": len(rq) - 1, "sha256_mod": digest(rq),
                       "at": {"0": digest([v[0]]), "1": digest([v[1]])}}
        print(f"cfg5 job {i}: {recs[i]['check']} (D = {D}), {time.time() - t0:.0f} s", flush=True)
    dt = time.time() - t0
    out = {"recipe": f"workloads.cfg5_stream(seed=1)[:{CFG5_JOBS}]; gcd jobs: oracle.gcd.gcd_z; "
                     f"resultant jobs: oracle.resultant.res_y if the degree bound is <= "
                     f"{CFG5_EXACT_MAX_D}, else res_y_modp mod 2^61 - 1 and the exact values at "
                     "x = 0 and x = 1 (oracle.resultant.res_at_point)",
           "digest": "sha256 of the coefficients (ascending) as comma-separated decimal "
                     "integers; 'at' digests one value the same way",
           "modulus": Q61, "oracle_seconds": round(dt, 1), "processes": procs, "jobs": recs}
    _write_json("cfg5_seed1_first32.json", out)
    return dt


def main():
    ap = argparse.ArgumentParser()
    ap.add_argument("--procs", type=int, default=os.cpu_count())
    ap.add_argument("--only", default="cfg2,cfg3,cfg4,cfg5,psc2")
    args = ap.parse_args()
    todo = args.only.split(",")
    ctx = mp.get_context("spawn")
    with ctx.Pool(args.procs) as pool:
        for name, fn in (("cfg2", make_cfg2), ("cfg3", make_cfg3), ("cfg4", make_cfg4),
                         ("cfg5", make_cfg5), ("psc2", make_psc_cfg2)):
            if name in todo:
                dt = fn(pool, args.procs)
                print(f"{name}: {dt:.1f} s", flush=True)


if __name__ == "__main__":
    main()
