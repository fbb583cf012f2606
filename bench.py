#!/usr/bin/env python
"""Benchmark of the exact bivariate resultant on GB300.

Workload: the discriminant-type resultant res_y(f, df/dy) of one dense random curve f of
total degree 32 with uniform signed 32-bit coefficients (seeded, synthetic).  One step is
one whole resultant: plan, reduction mod every prime, evaluation on each prime's point
set, the univariate resultants mod p, interpolation and mixed-radix reconstruction of
the integer coefficients.

``value`` is resultants per second over all ranks with device-resident inputs (CUDA
events on the library's stream, L2 flushed between steps outside the events); ``e2e``
is the same metric through the C ABI call with host buffers (copies included).

--impl reference times the CPU oracle (exact Bareiss determinants at integer points
plus exact interpolation) on the host cores: its timed steps together compute one whole
resultant of the same workload.  ``cpu_baseline`` in the main line is one whole oracle
resultant on all host cores, compared with the GPU's result.
"""

from __future__ import annotations

import argparse
import json
import os
import statistics
import subprocess
import sys
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = "exact res_y(f,g) in Z[x] per second"
UNIT = "resultants/s"
WORKLOAD = "res_y(f, df/dy), f dense total degree 32, signed 32-bit coefficients, seed 1"
SEED = 1
# DRAM bytes (read + write) of one k_unires<33> launch of this workload, from one ncu capture
# (caches flushed between passes, as ncu does)
K3_DRAM_BYTES = 21370368


def _args():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=50)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--no-extras", action="store_true",
                    help="skip the batched (4096 pairs) and served-stream measurements")
    ap.add_argument("--case", choices=sorted(CASES),
                    help="run one workload --reps times for a profiler instead of the benchmark")
    ap.add_argument("--reps", type=int, default=2)
    return ap.parse_args()


# --------------------------------------------------------------------------------------
# CPU oracle (reference arm and cpu_baseline)
# --------------------------------------------------------------------------------------

def _cpu_pool():
    import multiprocessing as mp
    cores = os.cpu_count() or 1
    return mp.get_context("spawn").Pool(cores), cores


def _oracle_points(f, g):
    """The integer points of the oracle's points route for res(f, g; y)."""
    from oracle.resultant import degree_bound
    D = degree_bound(f, g)
    x0 = -(D // 2)
    return x0, list(range(x0, x0 + D + 1))


def _oracle_whole(f, g, pool):
    """One whole oracle resultant: every exact point determinant on the pool, then the
    exact interpolation (oracle.resultant.res_y, points route).  Returns (R, seconds)."""
    from oracle.resultant import res_y
    t0 = time.perf_counter()
    r = res_y(f, g, route="points", map=lambda fn, xs: pool.map(fn, xs, chunksize=1))
    return r, time.perf_counter() - t0


def _cpu_baseline(f, g, pool, cores, want=None):
    """cpu_baseline of the main line: one whole resultant of the workload by the oracle on
    all host cores (no sampling, no extrapolation); checked against the GPU's result."""
    r, dt = _oracle_whole(f, g, pool)
    x0, xs = _oracle_points(f, g)
    out = {"value": 1.0 / dt, "unit": UNIT, "cores": cores, "kind": "oracle",
           "seconds": dt,
           "sample": f"one whole resultant: all {len(xs)} exact Bareiss point determinants "
                     f"(63x63 over Z) on {cores} processes and the exact interpolation"}
    if want is not None:
        out["equals_gpu_result"] = (r == want)
    return out


def run_reference(args):
    """The oracle as the reference arm: the K timed steps together compute one whole
    resultant of the workload (step s takes its share of the point determinants on all
    host cores; the last step also interpolates), so value = 1 resultant / the K steps'
    time; the W warm-up steps compute shares of the same size, untimed."""
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return
    from oracle.resultant import interpolate_consecutive, res_at_point
    from functools import partial
    from workloads import cfg2_pair
    f, g = cfg2_pair(SEED)
    pool, cores = _cpu_pool()
    x0, xs = _oracle_points(f, g)
    fn = partial(res_at_point, f, g)

    def shares(k):
        return [xs[i::k] for i in range(k)]

    parts = shares(args.steps)
    for w in range(args.warmup):             # untimed steps of the same size
        pool.map(fn, parts[w % len(parts)], chunksize=1)
    vals = {}
    step_s = []
    for s_i, part in enumerate(parts):
        t0 = time.perf_counter()
        vals.update(zip(part, pool.map(fn, part, chunksize=1)))
        if s_i == len(parts) - 1:
            r = interpolate_consecutive(x0, [vals[x] for x in xs])
        step_s.append(time.perf_counter() - t0)
    pool.close()
    total = sum(step_s)
    ms = 1000.0 * total / args.steps
    value = 1.0 / total
    line = {"impl": "reference", "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None, "dtype": "int64",
            "data": "synthetic", "config": {"workload": WORKLOAD, "m_y": 32, "n_y": 31,
                                           "D": len(xs) - 1,
                                           "resultants_per_step": 1.0 / args.steps},
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": cores, "kind": "oracle",
                             "seconds": total,
                             "sample": f"one whole resultant split over the {args.steps} timed "
                                       f"steps: its {len(xs)} exact point determinants on "
                                       f"{cores} processes, then the exact interpolation "
                                       f"(degree {len(r) - 1})"},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0, "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)


# --------------------------------------------------------------------------------------
# GPU arm
# --------------------------------------------------------------------------------------

class ClockSampler:
    FIELDS = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
              "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
              "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, gpu_index):
        self.gpu = gpu_index
        self.proc = None
        self.path = None

    def start(self):
        import tempfile
        self.path = tempfile.mktemp(suffix=".csv")
        try:
            self.proc = subprocess.Popen(
                ["nvidia-smi", f"--id={self.gpu}", f"--query-gpu={self.FIELDS}",
                 "--format=csv,noheader,nounits", "-lms", "100"],
                stdout=open(self.path, "w"), stderr=subprocess.DEVNULL)
        except Exception:
            self.proc = None

    def stop(self):
        if not self.proc:
            return {"sm_mhz": None, "sm_max_mhz": None, "reasons": ["unsampled"]}
        self.proc.terminate()
        try:
            self.proc.wait(timeout=5)
        except Exception:
            self.proc.kill()
        sm, smax, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for line in open(self.path):
            parts = [p.strip() for p in line.split(",")]
            if len(parts) < 9:
                continue
            try:
                sm.append(float(parts[1]))
                smax.append(float(parts[2]))
            except ValueError:
                continue
            for n, v in zip(names, parts[5:9]):
                if v.lower().startswith("active"):
                    reasons.add(n)
        os.unlink(self.path)
        return {"sm_mhz": statistics.median(sm) if sm else None,
                "sm_max_mhz": max(smax) if smax else None,
                "reasons": sorted(reasons), "samples": len(sm)}


def replica_step_ms(ms, dist, device):
    """Step time of a replicas-only run: the slowest rank's mean (max over ranks)."""
    import torch
    t = torch.tensor([float(ms)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return float(t.item())


def replica_value(ms, world):
    """Whole-job resultants per second: every rank computes one resultant per step."""
    return world * 1000.0 / ms


def _marshal_pairs(bs, pairs):
    """Pre-marshalled C arrays of a batch (kept alive by the returned tuple)."""
    import ctypes as C
    import numpy as np
    from paper_1201_1548_gb300._abi import _Bipoly, _Upoly
    n = len(pairs)
    keep = []
    F = (_Bipoly * n)()
    G = (_Bipoly * n)()
    for i, (f, g) in enumerate(pairs):
        af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
        keep += [af, ag]
        F[i] = _Bipoly(dxf, dyf, Lf, af.ctypes.data)
        G[i] = _Bipoly(dxg, dyg, Lg, ag.ctypes.data)
    O = (_Upoly * n)()
    for i in range(n):
        O[i] = _Upoly(0, 0, None)
    lib = bs.load_library()
    return F, G, O, keep, lib, C


def _bench_batched(bs, ctx, reps=3):
    """cfg3: 4096 pairs in one graph launch against one call per resultant, both through
    the C ABI with host buffers (plan, copies and formatting included)."""
    import numpy as np
    from workloads import cfg3_batch
    pairs = cfg3_batch(seed=1, count=4096)
    n = len(pairs)
    F, G, O, keep, lib, C = _marshal_pairs(bs, pairs)
    rc = lib.bs_resultant_batch(ctx.h, n, F, G, 1, O)          # size query
    if rc:
        raise SystemExit(f"size query failed: {rc}")
    caps = [(O[i].deg, O[i].limbs) for i in range(n)]
    bufs = [np.zeros((max(d, 0) + 1) * L, dtype=np.uint32) for d, L in caps]
    for i in range(n):
        O[i].c = bufs[i].ctypes.data

    def reset():
        for i in range(n):
            O[i].deg, O[i].limbs = caps[i]

    def batch_call():
        reset()
        t0 = time.perf_counter()
        rc = lib.bs_resultant_batch(ctx.h, n, F, G, 1, O)
        t1 = time.perf_counter()
        if rc:
            raise SystemExit(f"bs_resultant_batch failed: {rc}")
        return t1 - t0

    batch_call()                                                # warm-up (tables, graph)
    st = bs._abi._Stats()
    lib.bs_last_stats(ctx.h, C.byref(st))
    tb_default = min(batch_call() for _ in range(reps))
    # launch shapes autotuned on this batch (stage times by CUDA events), then timed again
    info = bs._abi._TuneInfo()
    rc = lib.bs_autotune_batch(ctx.h, n, F, G, 1, C.byref(info))
    if rc:
        raise SystemExit(f"bs_autotune_batch failed: {rc}")
    tune = {"eval_independent": info.eval_independent,
            "eval_warps": info.eval_warps, "eval_blocks_per_sm": info.eval_blocks_per_sm,
            "uni_threads": list(info.uni_threads), "crt_tile": info.crt_tile,
            "crt_blocks_per_sm": info.crt_blocks_per_sm, "trials": info.trials,
            "stage_ms_default": info.ms_default, "stage_ms_tuned": info.ms_tuned}
    batch_call()
    tb = min(batch_call() for _ in range(reps))
    ref = [bs.limbs_to_ints(bufs[i], O[i].deg + 1, O[i].limbs) if O[i].deg >= 0 else []
           for i in range(n)]
    # one blocking call (one launch sequence, no graph) per resultant
    one = (bs._abi._Upoly * n)()
    bufs1 = [np.zeros_like(b) for b in bufs]
    for i in range(n):
        one[i] = bs._abi._Upoly(caps[i][0], caps[i][1], bufs1[i].ctypes.data)
    for i in range(64):
        lib.bs_resultant(ctx.h, C.byref(F[i]), C.byref(G[i]), 1, C.byref(one[i]))
    for i in range(n):
        one[i].deg, one[i].limbs = caps[i]
    t0 = time.perf_counter()
    for i in range(n):
        rc = lib.bs_resultant(ctx.h, C.byref(F[i]), C.byref(G[i]), 1, C.byref(one[i]))
        if rc:
            raise SystemExit(f"bs_resultant failed: {rc}")
    t1 = (time.perf_counter() - t0)
    for i in range(0, n, 97):                                   # same results either way
        got = bs.limbs_to_ints(bufs1[i], one[i].deg + 1, one[i].limbs) if one[i].deg >= 0 else []
        if got != ref[i]:
            raise SystemExit(f"batched and single results differ at pair {i}")
    return {"workload": "4096 pairs, total degrees 4-24, 8-64-bit coefficients, 20% zeros, "
                        "seed 1 (host buffers, planning and copies included)",
            "pairs": n, "ms_batch": tb * 1e3, "ms_batch_default_shapes": tb_default * 1e3,
            "autotuned": tune, "ms_one_call_per_resultant": t1 * 1e3,
            "resultants_per_s_batch": n / tb, "resultants_per_s_one_by_one": n / t1,
            "speedup": t1 / tb, "instances": st.instances, "mulmods_alg": st.mulmods_alg,
            "modp_univariate_resultants_per_s": st.instances / tb}


def _bench_projection(bs, ctx, f, g, R, reps=3):
    """The projection steps after the resultant on the degree-32 curve (host buffers, one C
    call each, best of `reps` after a warm-up): the square-free part and Yun's
    factorisation of R = res(f, f_y), the 31 principal subresultant coefficients of f and
    f_y (exact and modulo one prime), and the fiber counts N (exact) and N^- (one prime)."""
    import ctypes as C
    import numpy as np
    lib = ctx.lib

    def best(fn):
        fn()
        out = []
        for _ in range(reps):
            t0 = time.perf_counter()
            fn()
            out.append(time.perf_counter() - t0)
        return min(out) * 1e3

    Ra, RL = bs.ints_to_limbs(R)
    Ru = bs._abi._Upoly(len(R) - 1, RL, Ra.ctypes.data)
    q = bs._abi._Upoly(0, 0, None)
    lib.bs_squarefree_part(ctx.h, C.byref(Ru), C.byref(q))
    sq_buf = np.zeros((q.deg + 1) * q.limbs, dtype=np.uint32)
    sq_cap = (q.deg, q.limbs)

    def sqf():
        o = bs._abi._Upoly(sq_cap[0], sq_cap[1], sq_buf.ctypes.data)
        if lib.bs_squarefree_part(ctx.h, C.byref(Ru), C.byref(o)):
            raise SystemExit("bs_squarefree_part failed")

    nf = np.zeros(1, dtype=np.int32)
    yq = bs._abi._Upoly(0, 0, None)
    lib.bs_squarefree_factorization(ctx.h, C.byref(Ru), 0, None, nf.ctypes.data, C.byref(yq))
    y_buf = np.zeros((yq.deg + 1) * yq.limbs, dtype=np.uint32)
    fdeg = np.zeros(max(int(nf[0]), 1), dtype=np.int32)
    y_cap = (yq.deg, yq.limbs, int(nf[0]))

    def yun():
        o = bs._abi._Upoly(y_cap[0], y_cap[1], y_buf.ctypes.data)
        if lib.bs_squarefree_factorization(ctx.h, C.byref(Ru), y_cap[2], fdeg.ctypes.data,
                                           nf.ctypes.data, C.byref(o)):
            raise SystemExit("bs_squarefree_factorization failed")

    af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
    fb, gb = bs._abi._bip(af, dxf, dyf, Lf), bs._abi._bip(ag, dxg, dyg, Lg)
    nq = C.c_int32(0)
    lib.bs_psc(ctx.h, C.byref(fb), C.byref(gb), 1, 0, C.byref(nq), None)
    n = nq.value
    outs = (bs._abi._Upoly * n)()
    for i in range(n):
        outs[i] = bs._abi._Upoly(0, 0, None)
    lib.bs_psc(ctx.h, C.byref(fb), C.byref(gb), 1, n, C.byref(nq), C.cast(outs, C.c_void_p))
    caps = [(outs[i].deg, outs[i].limbs) for i in range(n)]
    pbufs = [np.zeros((d + 1) * L, dtype=np.uint32) for d, L in caps]

    def psc():
        for i in range(n):
            outs[i] = bs._abi._Upoly(caps[i][0], caps[i][1], pbufs[i].ctypes.data)
        if lib.bs_psc(ctx.h, C.byref(fb), C.byref(gb), 1, n, C.byref(nq), C.cast(outs, C.c_void_p)):
            raise SystemExit("bs_psc failed")

    dmax, pp = C.c_int32(0), C.c_uint32(0)
    lib.bs_psc_modp(ctx.h, C.byref(fb), C.byref(gb), 1, C.byref(nq), C.byref(dmax), None, None,
                    C.byref(pp))
    mdeg = np.zeros(n, dtype=np.int32)
    mcoef = np.zeros(n * (dmax.value + 1), dtype=np.uint32)

    def psc_modp():
        if lib.bs_psc_modp(ctx.h, C.byref(fb), C.byref(gb), 1, C.byref(nq), C.byref(dmax),
                           mdeg.ctypes.data, mcoef.ctypes.data, C.byref(pp)):
            raise SystemExit("bs_psc_modp failed")

    degs = np.zeros(64, dtype=np.int32)
    s_, N_, p_ = C.c_int32(0), C.c_int64(0), C.c_uint32(0)
    counts = {}

    def fiber(mode):
        def run():
            if lib.bs_fiber_count(ctx.h, C.byref(fb), 1, mode, 64, degs.ctypes.data, C.byref(s_),
                                  C.byref(N_), C.byref(p_)):
                raise SystemExit("bs_fiber_count failed")
            counts[mode] = (int(N_.value), [int(x) for x in degs[: s_.value]])
        return run

    res = {"workload": "R = res(f, f_y), f dense total degree 32, signed 32-bit, seed 1 "
                       "(deg R = %d, host buffers)" % (len(R) - 1),
           "ms_squarefree_part": best(sqf), "ms_yun": best(yun), "ms_psc_exact": best(psc),
           "ms_psc_one_prime": best(psc_modp), "ms_fiber_count_exact": best(fiber(0)),
           "ms_fiber_lower_bound": best(fiber(1))}
    res["yun_factor_degrees"] = [int(x) for x in fdeg[: int(nf[0])]]
    res["psc_count"] = n
    res["fiber_N"], res["fiber_degs"] = counts[0]
    res["fiber_N_lower"] = counts[1][0]
    return res


def _bench_served(bs, jobs=96, seed=1):
    """cfg5: Poisson arrivals of resultant and gcd jobs (total degree 6-64, 16-256-bit
    coefficients) into the serving loop.  First a closed-loop pass (everything submitted
    at once) gives the saturated throughput; then an open-loop pass at 70% of it gives
    the latency percentiles."""
    from workloads import cfg5_stream
    srv = bs.Context(0)
    slots = 6  # three take any job, three no large ones
    srv.serve_start(slots=slots, max_batch=16)
    stream = cfg5_stream(seed=seed, jobs=jobs)

    def submit(job):
        if job["kind"] == "gcd":
            return srv.submit(bs.JOB_GCD, job["a"], job["b"])
        return srv.submit(bs.JOB_RESULTANT, job["f"], job["g"])

    warm = [submit(j) for j in stream[:8]]
    for t in warm:
        srv.wait(t)
        srv.poll(t)
    t0 = time.perf_counter()
    tickets = [submit(j) for j in stream]
    for t in tickets:
        srv.wait(t)
    sat_s = time.perf_counter() - t0
    for t in tickets:
        srv.poll(t)
    sat_rate = jobs / sat_s
    rate = 0.7 * sat_rate
    info0 = srv.serve_stats()
    stream2 = cfg5_stream(seed=seed + 1, jobs=jobs, rate_hz=rate)
    t0 = time.perf_counter()
    tickets = []
    for j in stream2:
        dt = j["t"] - (time.perf_counter() - t0)
        if dt > 0:
            time.sleep(dt)
        tickets.append(submit(j))
    lat, queue = [], []
    for t in tickets:
        srv.wait(t)
        status, _, qms, ms = srv.poll(t)
        if status:
            raise SystemExit(f"served job failed: {status}")
        lat.append(ms)
        queue.append(qms)
    open_s = time.perf_counter() - t0
    info = srv.serve_stats()
    srv.serve_stop()
    srv.close()

    def work_class(job):
        # the library's work classes: a resultant is large when its univariate stage
        # counts more than 2e9 multiply-reduce operations, tiny at most 2e8
        if job["kind"] == "gcd":
            return "gcd"
        p = bs.bs_plan(job["f"], job["g"])
        ops = p["k_total"] * p["N"] * p["m_e"] * p["n_e"]
        return "resultant_large" if ops > 2e9 else "resultant_small" if ops > 2e8 else "resultant_tiny"

    def pct_of(vals, q):
        vals = sorted(vals)
        return vals[min(len(vals) - 1, int(round(q * (len(vals) - 1))))]
    by_class, q_class = {}, {}
    for j, ms, qms in zip(stream2, lat, queue):
        by_class.setdefault(work_class(j), []).append(ms)
        q_class.setdefault(work_class(j), []).append(qms)
    classes = {k: {"jobs": len(v), "p50": pct_of(v, 0.5), "p99": pct_of(v, 0.99), "max": max(v),
                   "queue_p50": pct_of(q_class[k], 0.5), "queue_p99": pct_of(q_class[k], 0.99)}
               for k, v in sorted(by_class.items())}
    lat.sort()
    pct = lambda q: lat[min(len(lat) - 1, int(round(q * (len(lat) - 1))))]
    return {"workload": "Poisson stream, 50% resultants (dense, total degree 6-64) / 50% gcds "
                        f"(planted factor), 16-256-bit coefficients, seed {seed}",
            "jobs": jobs, "slots": slots, "max_batch": 16,
            "saturated_jobs_per_s": sat_rate, "offered_rate_hz": rate,
            "open_loop_jobs_per_s": jobs / open_s,
            "latency_ms": {"p50": pct(0.50), "p99": pct(0.99), "max": lat[-1]},
            "latency_ms_by_class": classes,
            "batches": info["batches"], "max_inflight_batches": info["max_inflight"],
            "arena_peak_bytes": info["arena_peak"],
            "open_loop_phase_ms": {k: info[k] - info0[k] for k in ("host_plan_ms", "device_ms", "host_finish_ms")}}


def run_ours(args):
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    pool = cores = None
    want_cpu = rank == 0 and world == 1 and not args.no_cpu_baseline
    if want_cpu:
        pool, cores = _cpu_pool()   # spawn before the first GPU call
    import numpy as np
    import torch
    torch.cuda.set_device(local)
    if world > 1:
        import torch.distributed as dist
        dist.init_process_group("nccl", device_id=torch.device("cuda", local))
    from paper_1201_1548_gb300.build import build
    if rank == 0:
        build()
    if world > 1:
        dist.barrier()
    import paper_1201_1548_gb300 as bs
    from paper_1201_1548_gb300._abi import _Bipoly, _Upoly
    import ctypes as C
    from workloads import cfg2_pair

    f, g = cfg2_pair(SEED)
    plan = bs.bs_plan(f, g)
    ctx = bs.Context(local)
    # a dedicated (non-default) stream shared by torch and the library, so that the CUDA
    # events below bracket exactly the library's work
    stream = torch.cuda.Stream()
    torch.cuda.set_stream(stream)
    ctx.set_stream(stream.cuda_stream)
    af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
    df = torch.from_numpy(af.view(np.int32).copy()).cuda()
    dg = torch.from_numpy(ag.view(np.int32).copy()).cuda()
    dcap, lcap = ctx.resultant_bounds((dxf, dyf, Lf), (dxg, dyg, Lg))
    out = torch.zeros((dcap + 1) * lcap, dtype=torch.int32, device="cuda")
    flush = torch.empty(256 << 20, dtype=torch.uint8, device="cuda")

    def step():
        ctx.resultant_device(df.data_ptr(), (dxf, dyf, Lf), dg.data_ptr(), (dxg, dyg, Lg),
                             out.data_ptr(), (dcap, lcap))

    # correctness guard outside timing: device path == host path
    host = ctx.resultant(f, g)
    step()
    ctx.device_status()
    dev = bs.limbs_to_ints(out.cpu().numpy().view(np.uint32), dcap + 1, lcap)
    while dev and dev[-1] == 0:
        dev.pop()
    if dev != host:
        raise SystemExit("device path and host path disagree")

    # per-stage device times from a separate profiled pass (the stage events separate the
    # kernels, so the timed steps below run without them)
    ctx.profile(True)
    stages = []
    for i in range(args.warmup + 10):
        flush.zero_()
        step()
        if i >= args.warmup:
            stages.append(ctx.stage_times())
    ctx.device_status()
    ctx.profile(False)
    for _ in range(args.warmup):
        flush.zero_()
        step()
    ctx.device_status()
    clocks = ClockSampler(local)
    if world > 1:
        dist.barrier()
    torch.cuda.synchronize()
    clocks.start()
    time.sleep(0.3)
    e0 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    e1 = [torch.cuda.Event(enable_timing=True) for _ in range(args.steps)]
    # after each flush a short device-side wait (about 50 us at 2 GHz), outside the events:
    # the host queues the whole step meanwhile, so the timed region holds the step's device
    # work without gaps where the GPU waits for a launch (the e2e figure carries the host
    # path: planning, launches, copies)
    for i in range(args.steps):
        flush.zero_()
        torch.cuda._sleep(100_000)
        e0[i].record(stream)
        step()
        e1[i].record(stream)
    torch.cuda.synchronize()
    if world > 1:
        dist.barrier()
    clk = clocks.stop()
    ctx.device_status()
    step_ms = [a.elapsed_time(b) for a, b in zip(e0, e1)]
    ms = statistics.mean(step_ms)
    if world > 1:
        ms = replica_step_ms(ms, dist, torch.device("cuda", local))
    value = replica_value(ms, world)
    srt = sorted(step_ms)
    p50 = srt[len(srt) // 2]
    p99 = srt[min(len(srt) - 1, int(round(0.99 * (len(srt) - 1))))]
    k3 = statistics.mean(s[2] for s in stages)
    stage_avg = [statistics.mean(s[i] for s in stages) for i in range(5)]
    instances = plan["k_total"] * plan["N"]
    m_e, n_e = plan["m_e"], plan["n_e"]
    # dominant kernel: the univariate-resultant stage (ALU bound)
    alg_mulmods = instances * m_e * n_e
    achieved = alg_mulmods / (k3 * 1e-3) / 1e9
    clk_probe = ClockSampler(local)
    clk_probe.start()
    probe = {k: ctx.alu_probe(i) / 1e12 for i, k in
             enumerate(("mad_lo_Tops", "mad_hi_Tops", "mad_wide_Tops", "mulmod_Tops"))}
    probe["clock_mhz"] = clk_probe.stop().get("sm_mhz") or 2070.0
    import torch.cuda as tc
    props = tc.get_device_properties(local)
    sms = props.multi_processor_count
    max_mhz = clk.get("sm_max_mhz") or 2070.0
    # peaks of the integer multiply pipe for one Montgomery multiplication (one mad.wide,
    # one mad.lo, one mad.hi), from the per-SM-per-clock rates of those instructions that
    # the probe measures, times SMs and the maximum clock
    probe_mhz = probe.pop("clock_mhz")
    per_clk = {k: probe[k] * 1e12 / (sms * probe_mhz * 1e6)
               for k in ("mad_lo_Tops", "mad_hi_Tops", "mad_wide_Tops")}
    mix = 1.0 / (1.0 / per_clk["mad_wide_Tops"] + 1.0 / per_clk["mad_lo_Tops"]
                 + 1.0 / per_clk["mad_hi_Tops"])
    peak = sms * max_mhz * 1e6 * mix / 1e9
    # four multiplications at the full low-product rate (64 per SM per clock)
    peak_lo = sms * max_mhz * 1e6 * 64 / 4 / 1e9
    roof = {"bound": "alu", "achieved": achieved, "peak": peak, "unit": "Gmulmod/s",
            "frac": achieved / peak, "traffic": K3_DRAM_BYTES,
            "kernel": "k_unires<33>", "alg_per_launch": alg_mulmods,
            "peak_basis": "measured mad.wide + mad.lo + mad.hi rates per SM and clock "
                          f"({mix:.2f} Montgomery multiplications per SM per clock) x "
                          f"{sms} SMs x {max_mhz:.0f} MHz",
            "peak_lo_rate": peak_lo, "frac_vs_lo_rate": achieved / peak_lo,
            "note": "algorithmic m_e*n_e mulmods per (prime, point) instance"}

    # e2e through the C ABI with pinned host buffers
    hf = torch.from_numpy(af.view(np.int32).copy()).pin_memory()
    hg = torch.from_numpy(ag.view(np.int32).copy()).pin_memory()
    pdeg = plan["D"]
    hout = torch.zeros((pdeg + 1) * plan["out_limbs"], dtype=torch.int32).pin_memory()
    fb = _Bipoly(dxf, dyf, Lf, hf.data_ptr())
    gb = _Bipoly(dxg, dyg, Lg, hg.data_ptr())
    lib = bs.load_library()

    def e2e_call():
        ob = _Upoly(pdeg, plan["out_limbs"], hout.data_ptr())
        rc = lib.bs_resultant(ctx.h, C.byref(fb), C.byref(gb), 1, C.byref(ob))
        if rc:
            raise SystemExit(f"bs_resultant failed: {rc}")
        return ob.deg

    for _ in range(args.warmup):
        e2e_call()
    torch.cuda.synchronize()
    e2e_total = 0.0
    for _ in range(args.steps):
        flush.zero_()                      # L2 flush between calls, outside the timing
        torch.cuda.synchronize()
        t0 = time.perf_counter()
        deg = e2e_call()                   # upload, stages, download, formatting
        e2e_total += time.perf_counter() - t0
    e2e_s = e2e_total / args.steps
    e2e_val = world * 1.0 / e2e_s
    h2d = (af.nbytes + ag.nbytes)
    d2h = (deg + 1) * plan["out_limbs"] * 4

    batched = served = projection = None
    if rank == 0 and not args.no_extras:
        # the extra measurements never cost the headline line: a failure is reported in it
        def extra(fn):
            try:
                return fn()
            except (Exception, SystemExit) as e:  # noqa: BLE001
                return {"error": f"{type(e).__name__}: {e}"}
        batched = extra(lambda: _bench_batched(bs, ctx))
        served = extra(lambda: _bench_served(bs))
        projection = extra(lambda: _bench_projection(bs, ctx, f, g, ctx.resultant(f, g)))

    cpu = None
    if want_cpu:
        cpu = _cpu_baseline(f, g, pool, cores, want=host)
        pool.close()
    if rank == 0:
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": ms,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "u32", "data": "synthetic",
                "config": {"workload": WORKLOAD, "m_y": m_e, "n_y": n_e, "D": plan["D"],
                           "points_per_prime": plan["N"], "primes": plan["k_need"],
                           "primes_evaluated": plan["k_total"],
                           "l2": "flushed between steps (256 MiB write, outside the events)",
                           "launch_headroom": "a 100k-cycle device wait after each flush, outside the events",
                           "parallelism": "replicas" if world > 1 else "single"},
                "latency_ms": {"p50": p50, "p99": p99},
                "modp_univariate_resultants_per_s": world * instances / (ms * 1e-3),
                "stage_ms": dict(zip(("plan", "reduce_eval", "unires", "interp", "crt"), stage_avg)),
                "roofline": roof, "alu_probe": probe, "clocks": clk,
                "e2e": {"value": e2e_val, "unit": UNIT, "h2d_bytes_per_step": h2d,
                        "d2h_bytes_per_step": d2h},
                "gpu_launches": 6 * args.steps,
                "cpu_baseline": cpu,
                "batched": batched, "served": served, "projection": projection}
        print(json.dumps(line), flush=True)
    ctx.close()
    if world > 1:
        dist.destroy_process_group()


# --------------------------------------------------------------------------------------
# single workloads for profilers (--case): each repetition is one call; the result is
# checked once against the host entry point
# --------------------------------------------------------------------------------------

def _case_discriminant32(reps):
    """res_y(f, df/dy) of the degree-32 curve with device-resident inputs, one
    bs_resultant_device call per repetition."""
    import numpy as np
    import torch
    import paper_1201_1548_gb300 as bs
    from workloads import cfg2_pair
    f, g = cfg2_pair(SEED)
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


def _case_batch4096(reps):
    """The 4096 ragged pairs through bs_resultant_batch, one graph launch per repetition."""
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


def _case_projection32(reps):
    """Square-free part, Yun's factorisation and the psc sequence of R = res(f, f_y) for
    the degree-32 curve, one call each per repetition."""
    import paper_1201_1548_gb300 as bs
    from workloads import cfg2_pair
    f, g = cfg2_pair(SEED)
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


def _case_large64(reps):
    """A degree 57 x 64 pair of dense curves with 256-bit coefficients (seed 7; 1,047
    primes x 4096 points), one bs_resultant call per repetition with the stages separated
    by events; prints each call's stage times."""
    import numpy as np
    import paper_1201_1548_gb300 as bs
    from workloads import dense_curve
    rng = np.random.Generator(np.random.PCG64(7))
    f = dense_curve(rng, 57, 256)
    g = dense_curve(rng, 64, 256)
    ctx = bs.Context(0)
    first = ctx.resultant(f, g)
    ctx.profile(True)
    for _ in range(reps):
        if ctx.resultant(f, g) != first:
            raise SystemExit("repeated calls differ")
        st = ctx.stage_times()
        print("stage ms (upload, evaluation, univariate, interpolation, reconstruction):",
              " ".join(f"{x:.3f}" for x in st))
    ctx.profile(False)
    print("stats", ctx.last_stats())


CASES = {"discriminant32": _case_discriminant32, "batch4096": _case_batch4096,
         "projection32": _case_projection32, "large64": _case_large64}


def run_case(args):
    from paper_1201_1548_gb300.build import build
    build()
    CASES[args.case](args.reps)
    print("ok")


def main():
    args = _args()
    if args.case:
        run_case(args)
        return
    if args.impl == "reference":
        run_reference(args)
    else:
        run_ours(args)


if __name__ == "__main__":
    main()
