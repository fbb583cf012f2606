"""ctypes binding of libbsres.so (argument marshalling only)."""

from __future__ import annotations

import ctypes as C
import os

import numpy as np

_HERE = os.path.dirname(os.path.abspath(__file__))
# BSRES_DEBUG=1 selects the build whose kernels bounds-check their accesses
_LIB_PATH = os.path.join(_HERE, "libbsres_debug.so" if os.environ.get("BSRES_DEBUG") == "1"
                         else "libbsres.so")
_LIB = None

# every symbol that include/bsres.h declares
EXPORTED_SYMBOLS = [
    "bs_init", "bs_free", "bs_set_stream", "bs_error_string", "bs_last_error_detail",
    "bs_last_stats", "bs_resultant_bounds", "bs_resultant", "bs_resultant_device",
    "bs_device_status", "bs_resultant_batch", "bs_uni_resultant_modp", "bs_prime_table",
    "bs_gcd_modp", "bs_squarefree_part", "bs_plan", "bs_alu_probe", "bs_profile",
    "bs_stage_times", "bs_resultant_device_noalloc", "bs_gcd_z", "bs_modgcd_batch",
    "bs_autotune_batch", "bs_set_tune", "bs_serve_start", "bs_serve_stop", "bs_submit", "bs_poll", "bs_wait", "bs_serve_stats",
    "bs_squarefree_factorization", "bs_squarefree_factorization_batch", "bs_psc",
    "bs_psc_modp", "bs_fiber_count", "bs_content", "bs_teissier_q", "bs_root_multiplicity",
    "bs_subresultant", "bs_gcd_bivariate",
]


class _TuneInfo(C.Structure):
    _fields_ = [("eval_warps", C.c_int32), ("eval_blocks_per_sm", C.c_int32),
                ("uni_threads", C.c_int32 * 6), ("crt_tile", C.c_int32),
                ("crt_blocks_per_sm", C.c_int32), ("ms_default", C.c_float),
                ("ms_tuned", C.c_float), ("trials", C.c_int32), ("eval_independent", C.c_int32)]


class BsError(RuntimeError):
    def __init__(self, code, msg):
        super().__init__(f"bsres error {code}: {msg}")
        self.code = code


class _Bipoly(C.Structure):
    _fields_ = [("deg_x", C.c_int32), ("deg_y", C.c_int32), ("limbs", C.c_int32),
                ("c", C.c_void_p)]


class _Upoly(C.Structure):
    _fields_ = [("deg", C.c_int32), ("limbs", C.c_int32), ("c", C.c_void_p)]


class _PlanInfo(C.Structure):
    _fields_ = [("trivial", C.c_int32), ("m_e", C.c_int32), ("n_e", C.c_int32),
                ("D", C.c_int32), ("N", C.c_int32), ("k_need", C.c_int32),
                ("k_total", C.c_int32), ("out_limbs", C.c_int32), ("log2B_q16", C.c_int64)]


class _Stats(C.Structure):
    _fields_ = [("jobs", C.c_int32), ("primes_needed", C.c_int64),
                ("primes_evaluated", C.c_int64), ("primes_rejected", C.c_int64),
                ("instances", C.c_int64), ("mulmods_alg", C.c_int64),
                ("max_points", C.c_int32), ("max_primes", C.c_int32)]


class _Job(C.Structure):
    _fields_ = [("kind", C.c_int32), ("var", C.c_int32), ("f", _Bipoly), ("g", _Bipoly),
                ("a", _Upoly), ("b", _Upoly)]


class _Result(C.Structure):
    _fields_ = [("status", C.c_int32), ("deg", C.c_int32), ("limbs", C.c_int32),
                ("c", C.c_void_p), ("cap_words", C.c_int64), ("queue_ms", C.c_double),
                ("latency_ms", C.c_double)]


class _ServeInfo(C.Structure):
    _fields_ = [("submitted", C.c_int64), ("completed", C.c_int64), ("batches", C.c_int64),
                ("jobs_in_batches", C.c_int64), ("queued", C.c_int64),
                ("inflight", C.c_int32), ("max_inflight", C.c_int32),
                ("arena_bytes", C.c_int64), ("arena_used", C.c_int64), ("arena_peak", C.c_int64),
                ("host_plan_ms", C.c_double), ("device_ms", C.c_double), ("host_finish_ms", C.c_double)]


BS_PENDING = 10
# status codes of include/bsres.h
(BS_OK, BS_ERR_ARG, BS_ERR_NOMEM, BS_ERR_UNLUCKY, BS_ERR_TIMEOUT, BS_ERR_CUDA, BS_ERR_ZERO,
 BS_ERR_RANGE, BS_ERR_INTERNAL, BS_ERR_CAPACITY) = range(10)
JOB_RESULTANT, JOB_GCD, JOB_SQFREE = 0, 1, 2


def library_path():
    return _LIB_PATH


def load_library():
    """Load libbsres.so; raise if it has not been built (no fallback path exists)."""
    global _LIB
    if _LIB is not None:
        return _LIB
    if not os.path.exists(_LIB_PATH):
        raise BsError(-1, f"{_LIB_PATH} is missing: build it with "
                          "`python -m paper_1201_1548_gb300.build`")
    lib = C.CDLL(_LIB_PATH)
    P = C.c_void_p
    I = C.c_int
    lib.bs_init.argtypes = [I, C.c_size_t, C.POINTER(P)]
    lib.bs_free.argtypes = [P]
    lib.bs_free.restype = None
    lib.bs_set_stream.argtypes = [P, P]
    lib.bs_error_string.argtypes = [I]
    lib.bs_error_string.restype = C.c_char_p
    lib.bs_last_error_detail.argtypes = [P]
    lib.bs_last_error_detail.restype = C.c_char_p
    lib.bs_last_stats.argtypes = [P, C.POINTER(_Stats)]
    lib.bs_resultant_bounds.argtypes = [C.POINTER(_Bipoly), C.POINTER(_Bipoly), I,
                                        C.POINTER(C.c_int32), C.POINTER(C.c_int32)]
    lib.bs_resultant.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I, C.POINTER(_Upoly)]
    lib.bs_resultant_device.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I,
                                        C.POINTER(_Upoly)]
    lib.bs_device_status.argtypes = [P]
    lib.bs_resultant_device_noalloc.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I,
                                                C.POINTER(_Upoly)]
    lib.bs_resultant_batch.argtypes = [P, I, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I,
                                       C.POINTER(_Upoly)]
    lib.bs_uni_resultant_modp.argtypes = [P, I, P, P, I, I, P, I, I, P]
    lib.bs_prime_table.argtypes = [I, P]
    lib.bs_gcd_modp.argtypes = [P, P, I, P, I, C.c_uint32, P, C.POINTER(C.c_int)]
    lib.bs_squarefree_part.argtypes = [P, C.POINTER(_Upoly), C.POINTER(_Upoly)]
    lib.bs_alu_probe.argtypes = [P, I, C.POINTER(C.c_double)]
    lib.bs_profile.argtypes = [P, I]
    lib.bs_stage_times.argtypes = [P, P, I]
    lib.bs_plan.argtypes = [C.POINTER(_Bipoly), C.POINTER(_Bipoly), I, C.POINTER(_PlanInfo)]
    lib.bs_gcd_z.argtypes = [P, C.POINTER(_Upoly), C.POINTER(_Upoly), C.POINTER(_Upoly)]
    lib.bs_autotune_batch.argtypes = [P, I, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I,
                                      C.POINTER(_TuneInfo)]
    lib.bs_set_tune.argtypes = [P, C.POINTER(_TuneInfo)]
    lib.bs_modgcd_batch.argtypes = [P, I, P, P, P, P]
    lib.bs_squarefree_factorization.argtypes = [P, C.POINTER(_Upoly), I, P, P, C.POINTER(_Upoly)]
    lib.bs_squarefree_factorization_batch.argtypes = [P, I, P, I, P, P, P]
    lib.bs_psc.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I, I, C.POINTER(C.c_int32), P]
    lib.bs_psc_modp.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I, C.POINTER(C.c_int32),
                                C.POINTER(C.c_int32), P, P, C.POINTER(C.c_uint32)]
    lib.bs_content.argtypes = [P, C.POINTER(_Bipoly), I, C.POINTER(_Upoly), I, P, C.POINTER(C.c_int32)]
    lib.bs_teissier_q.argtypes = [P, C.POINTER(_Bipoly), I, C.POINTER(_Upoly), C.POINTER(C.c_int32)]
    lib.bs_subresultant.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I, I, I,
                                    C.POINTER(C.c_int32), P]
    lib.bs_gcd_bivariate.argtypes = [P, C.POINTER(_Bipoly), C.POINTER(_Bipoly), I, I, P,
                                     C.POINTER(C.c_int32)]
    lib.bs_root_multiplicity.argtypes = [P, C.POINTER(_Upoly), C.POINTER(_Upoly), I, P, P,
                                         C.POINTER(_Upoly)]
    lib.bs_fiber_count.argtypes = [P, C.POINTER(_Bipoly), I, I, I, P, C.POINTER(C.c_int32),
                                   C.POINTER(C.c_int64), C.POINTER(C.c_uint32)]
    lib.bs_serve_start.argtypes = [P, I, I, C.c_size_t]
    lib.bs_serve_stop.argtypes = [P]
    lib.bs_submit.argtypes = [P, C.POINTER(_Job), C.POINTER(C.c_uint64)]
    lib.bs_poll.argtypes = [P, C.c_uint64, C.POINTER(_Result)]
    lib.bs_wait.argtypes = [P, C.c_uint64, I]
    lib.bs_serve_stats.argtypes = [P, C.POINTER(_ServeInfo)]
    for name in EXPORTED_SYMBOLS:
        getattr(lib, name)
    _LIB = lib
    return lib


# --------------------------------------------------------------------------------------
# marshalling
# --------------------------------------------------------------------------------------

def _limbs_for(values):
    bits = 1
    for v in values:
        b = (v if v >= 0 else ~v).bit_length() + 1
        if b > bits:
            bits = b
    return max(1, (bits + 31) // 32)


def ints_to_limbs(values, limbs=None):
    """Python ints -> (n, limbs) uint32 array of two's complement little-endian limbs."""
    values = [int(v) for v in values]
    L = limbs or _limbs_for(values)
    mask = (1 << (32 * L)) - 1
    raw = b"".join((v & mask).to_bytes(4 * L, "little") for v in values)
    arr = np.frombuffer(raw, dtype="<u4").reshape(len(values), L) if values else \
        np.zeros((0, L), dtype=np.uint32)
    return np.ascontiguousarray(arr, dtype=np.uint32), L


def limbs_to_ints(arr, ncoef, limbs):
    a = np.ascontiguousarray(np.asarray(arr, dtype=np.uint32).reshape(-1)[: ncoef * limbs])
    b = a.tobytes()
    w = 4 * limbs
    return [int.from_bytes(b[i * w:(i + 1) * w], "little", signed=True) for i in range(ncoef)]


def bipoly_to_limbs(f, limbs=None):
    """Grid f[j][i] (coefficient of x^i y^j) -> (uint32 array (deg_y+1, deg_x+1, L), dx, dy, L)."""
    dy = len(f) - 1
    dx = max(len(r) for r in f) - 1
    flat = []
    for row in f:
        flat.extend(row)
        flat.extend([0] * (dx + 1 - len(row)))
    arr, L = ints_to_limbs(flat, limbs)
    return arr.reshape(dy + 1, dx + 1, L), dx, dy, L


def _bip(arr, dx, dy, L):
    return _Bipoly(dx, dy, L, arr.ctypes.data)


class Context:
    """A library context on one CUDA device (owns device memory and a stream)."""

    def __init__(self, device=0, mem_budget=0):
        self.lib = load_library()
        h = C.c_void_p()
        rc = self.lib.bs_init(int(device), int(mem_budget), C.byref(h))
        if rc != 0:
            raise BsError(rc, self.lib.bs_error_string(rc).decode())
        self.h = h

    def close(self):
        if getattr(self, "h", None):
            self.lib.bs_free(self.h)
            self.h = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass

    def __enter__(self):
        return self

    def __exit__(self, *a):
        self.close()

    def _check(self, rc):
        if rc != 0:
            detail = self.lib.bs_last_error_detail(self.h).decode()
            raise BsError(rc, f"{self.lib.bs_error_string(rc).decode()} ({detail})")

    def set_stream(self, stream_ptr):
        self._check(self.lib.bs_set_stream(self.h, C.c_void_p(stream_ptr or None)))

    def last_stats(self):
        s = _Stats()
        self._check(self.lib.bs_last_stats(self.h, C.byref(s)))
        return {k: getattr(s, k) for k, _ in _Stats._fields_}

    # -- resultants -----------------------------------------------------------------
    def resultant(self, f, g, var=1):
        """res(f, g; y) (var=1) or res(f, g; x) (var=0) as a list of Python ints."""
        return self.resultant_batch([(f, g)], var=var, graph=False)[0]

    def psc(self, f, g, var=1):
        """[sr_0, ..., sr_(q-1)] of f and g with respect to y (var=1) or x (var=0), each a list
        of Python ints ([] for the zero polynomial)."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bipoly_to_limbs(g)
        fb, gb = _bip(af, dxf, dyf, Lf), _bip(ag, dxg, dyg, Lg)
        q = C.c_int32(0)
        self._check(self.lib.bs_psc(self.h, C.byref(fb), C.byref(gb), int(var), 0, C.byref(q), None))
        n = q.value
        if n == 0:
            return []
        outs = (_Upoly * n)()
        for i in range(n):
            outs[i] = _Upoly(0, 0, None)
        self._check(self.lib.bs_psc(self.h, C.byref(fb), C.byref(gb), int(var), n, C.byref(q),
                                    C.cast(outs, C.c_void_p)))
        bufs = []
        for i in range(n):
            buf = np.zeros((max(outs[i].deg, 0) + 1) * outs[i].limbs, dtype=np.uint32)
            bufs.append(buf)
            outs[i] = _Upoly(max(outs[i].deg, 0), outs[i].limbs, buf.ctypes.data)
        self._check(self.lib.bs_psc(self.h, C.byref(fb), C.byref(gb), int(var), n, C.byref(q),
                                    C.cast(outs, C.c_void_p)))
        return [limbs_to_ints(bufs[i], outs[i].deg + 1, outs[i].limbs) if outs[i].deg >= 0 else []
                for i in range(n)]

    def _rows_call(self, call, n):
        """The two-call pattern of an entry point writing n caller-owned rows: a size query,
        then the computation; returns the rows as lists of Python ints."""
        if n == 0:
            return []
        outs = (_Upoly * n)()
        for i in range(n):
            outs[i] = _Upoly(0, 0, None)
        self._check(call(n, C.cast(outs, C.c_void_p)))
        bufs = []
        for i in range(n):
            buf = np.zeros((max(outs[i].deg, 0) + 1) * outs[i].limbs, dtype=np.uint32)
            bufs.append(buf)
            outs[i] = _Upoly(max(outs[i].deg, 0), outs[i].limbs, buf.ctypes.data)
        self._check(call(n, C.cast(outs, C.c_void_p)))
        return [limbs_to_ints(bufs[i], outs[i].deg + 1, outs[i].limbs) if outs[i].deg >= 0 else []
                for i in range(n)]

    def subresultant(self, f, g, d, var=1):
        """[s_0, ..., s_d]: the d-th subresultant polynomial of f and g with respect to y
        (var=1) or x (var=0), s_j the coefficient of the j-th power (lists of Python ints)."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bipoly_to_limbs(g)
        fb, gb = _bip(af, dxf, dyf, Lf), _bip(ag, dxg, dyg, Lg)
        n = C.c_int32(0)
        self._check(self.lib.bs_subresultant(self.h, C.byref(fb), C.byref(gb), int(var), int(d), 0,
                                             C.byref(n), None))
        return self._rows_call(lambda cap, outs: self.lib.bs_subresultant(
            self.h, C.byref(fb), C.byref(gb), int(var), int(d), cap, C.byref(n), outs), n.value)

    def gcd_bivariate(self, f, g, var=1):
        """gcd(f, g) in Z[x, y] as rows by powers of y (var=1) or x (var=0), each a list of
        Python ints in the other variable ([] for gcd(0, 0))."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bipoly_to_limbs(g)
        fb, gb = _bip(af, dxf, dyf, Lf), _bip(ag, dxg, dyg, Lg)
        n = C.c_int32(0)
        self._check(self.lib.bs_gcd_bivariate(self.h, C.byref(fb), C.byref(gb), int(var), 0, None,
                                              C.byref(n)))
        return self._rows_call(lambda cap, outs: self.lib.bs_gcd_bivariate(
            self.h, C.byref(fb), C.byref(gb), int(var), cap, outs, C.byref(n)), n.value)

    def psc_modp(self, f, g, var=1):
        """(p, [sr_0 mod p, ...]) for the first accepted table prime p (ascending residues)."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bipoly_to_limbs(g)
        fb, gb = _bip(af, dxf, dyf, Lf), _bip(ag, dxg, dyg, Lg)
        q, dmax, p = C.c_int32(0), C.c_int32(0), C.c_uint32(0)
        self._check(self.lib.bs_psc_modp(self.h, C.byref(fb), C.byref(gb), int(var), C.byref(q),
                                         C.byref(dmax), None, None, C.byref(p)))
        n = q.value
        if n == 0:
            return 0, []
        deg = np.zeros(n, dtype=np.int32)
        coef = np.zeros(n * (dmax.value + 1), dtype=np.uint32)
        self._check(self.lib.bs_psc_modp(self.h, C.byref(fb), C.byref(gb), int(var), C.byref(q),
                                         C.byref(dmax), deg.ctypes.data, coef.ctypes.data, C.byref(p)))
        w = dmax.value + 1
        return int(p.value), [[int(x) for x in coef[i * w: i * w + int(deg[i]) + 1]] for i in range(n)]

    def content(self, f, var=1):
        """(h, rows): the content of f with respect to y (var=1) or x (var=0) and the rows of
        the primitive part f / h, ascending integer lists ([] for zero)."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        fb = _bip(af, dxf, dyf, Lf)
        n = (dyf if var else dxf) + 1
        h = _Upoly(0, 0, None)
        rows = (_Upoly * n)()
        for i in range(n):
            rows[i] = _Upoly(0, 0, None)
        nr = C.c_int32(0)
        self._check(self.lib.bs_content(self.h, C.byref(fb), int(var), C.byref(h), n,
                                         C.cast(rows, C.c_void_p), C.byref(nr)))
        hb = np.zeros((h.deg + 1) * h.limbs, dtype=np.uint32)
        h = _Upoly(h.deg, h.limbs, hb.ctypes.data)
        bufs = []
        for i in range(nr.value):
            bufs.append(np.zeros((rows[i].deg + 1) * rows[i].limbs, dtype=np.uint32))
            rows[i] = _Upoly(rows[i].deg, rows[i].limbs, bufs[i].ctypes.data)
        self._check(self.lib.bs_content(self.h, C.byref(fb), int(var), C.byref(h), nr.value,
                                         C.cast(rows, C.c_void_p), C.byref(nr)))
        conv = lambda u, b: limbs_to_ints(b, u.deg + 1, u.limbs) if u.deg >= 0 else []
        return conv(h, hb), [conv(rows[i], bufs[i]) for i in range(nr.value)]

    def teissier_q(self, f, var=1):
        """(Q, d): Teissier's Q = res(f_x / h, f_y / h; y) exactly, h = gcd(f_x, f_y) in
        Z[x, y] and d = deg_y h (x and y exchanged for var=0)."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        fb = _bip(af, dxf, dyf, Lf)
        q, d = _Upoly(0, 0, None), C.c_int32(0)
        self._check(self.lib.bs_teissier_q(self.h, C.byref(fb), int(var), C.byref(q), C.byref(d)))
        buf = np.zeros((max(q.deg, 0) + 1) * q.limbs, dtype=np.uint32)
        q = _Upoly(max(q.deg, 0), q.limbs, buf.ctypes.data)
        self._check(self.lib.bs_teissier_q(self.h, C.byref(fb), int(var), C.byref(q), C.byref(d)))
        return (limbs_to_ints(buf, q.deg + 1, q.limbs) if q.deg >= 0 else []), int(d.value)

    def root_multiplicity(self, r, q):
        """[c_0, c_1, ..., c_t]: the square-free part of the ascending integer list r split
        by the multiplicity of q at its roots (c_k vanishes exactly where q has multiplicity
        k), each primitive with a positive leading coefficient."""
        ar, Lr = ints_to_limbs(r)
        aq, Lq = ints_to_limbs(q)
        rb = _Upoly(len(r) - 1, Lr, ar.ctypes.data)
        qb = _Upoly(len(q) - 1, Lq, aq.ctypes.data)
        out, nfac = _Upoly(0, 0, None), C.c_int32(0)
        self._check(self.lib.bs_root_multiplicity(self.h, C.byref(rb), C.byref(qb), 0, None,
                                                  C.addressof(nfac), C.byref(out)))
        cap = max(int(nfac.value), 1)
        fdeg = np.zeros(cap, dtype=np.int32)
        buf = np.zeros((out.deg + 1) * out.limbs, dtype=np.uint32)
        out = _Upoly(out.deg, out.limbs, buf.ctypes.data)
        self._check(self.lib.bs_root_multiplicity(self.h, C.byref(rb), C.byref(qb), cap,
                                                  fdeg.ctypes.data, C.addressof(nfac),
                                                  C.byref(out)))
        coefs = limbs_to_ints(buf, out.deg + 1, out.limbs)
        facs, pos = [], 0
        for d in fdeg[: int(nfac.value)]:
            facs.append(coefs[pos: pos + int(d) + 1])
            pos += int(d) + 1
        return facs

    def fiber_count(self, f, var=1, mode=0):
        """(degs, N, p): deg R_1, deg R_2, ... of the decomposition of R* by fibers, the point
        count N (mode 0, exact), its lower bound N^- (mode 1) or upper bound N^+ (mode 2, no
        degrees) for one prime p."""
        af, dxf, dyf, Lf = bipoly_to_limbs(f)
        fb = _bip(af, dxf, dyf, Lf)
        cap = max(dxf, dyf) + 2
        degs = np.zeros(cap, dtype=np.int32)
        s, N, p = C.c_int32(0), C.c_int64(0), C.c_uint32(0)
        self._check(self.lib.bs_fiber_count(self.h, C.byref(fb), int(var), int(mode), cap,
                                            degs.ctypes.data, C.byref(s), C.byref(N), C.byref(p)))
        return [int(x) for x in degs[: s.value]], int(N.value), int(p.value)

    def resultant_batch(self, pairs, var=1, graph=True):
        n = len(pairs)
        keep = []
        fs = (_Bipoly * n)()
        gs = (_Bipoly * n)()
        for i, (f, g) in enumerate(pairs):
            af, dxf, dyf, Lf = bipoly_to_limbs(f)
            ag, dxg, dyg, Lg = bipoly_to_limbs(g)
            keep += [af, ag]
            fs[i] = _bip(af, dxf, dyf, Lf)
            gs[i] = _bip(ag, dxg, dyg, Lg)
        outs = (_Upoly * n)()
        for i in range(n):
            outs[i] = _Upoly(0, 0, None)
        fn = self.lib.bs_resultant_batch if graph else self.lib.bs_resultant
        if graph:
            self._check(fn(self.h, n, fs, gs, int(var), outs))
        else:
            for i in range(n):
                self._check(fn(self.h, C.byref(fs[i]), C.byref(gs[i]), int(var), C.byref(outs[i])))
        bufs = []
        for i in range(n):
            deg, L = outs[i].deg, outs[i].limbs
            buf = np.zeros((max(deg, 0) + 1) * L, dtype=np.uint32)
            bufs.append(buf)
            outs[i] = _Upoly(max(deg, 0), L, buf.ctypes.data)
        if graph:
            self._check(fn(self.h, n, fs, gs, int(var), outs))
        else:
            for i in range(n):
                self._check(fn(self.h, C.byref(fs[i]), C.byref(gs[i]), int(var), C.byref(outs[i])))
        res = []
        for i in range(n):
            deg, L = outs[i].deg, outs[i].limbs
            res.append(limbs_to_ints(bufs[i], deg + 1, L) if deg >= 0 else [])
        return res

    def resultant_bounds(self, f_meta, g_meta, var=1):
        """f_meta = (deg_x, deg_y, limbs); returns (deg_cap, limbs_cap)."""
        fb = _Bipoly(f_meta[0], f_meta[1], f_meta[2], None)
        gb = _Bipoly(g_meta[0], g_meta[1], g_meta[2], None)
        d = C.c_int32()
        L = C.c_int32()
        rc = self.lib.bs_resultant_bounds(C.byref(fb), C.byref(gb), int(var), C.byref(d), C.byref(L))
        self._check(rc)
        return d.value, L.value

    def resultant_device(self, f_ptr, f_meta, g_ptr, g_meta, out_ptr, out_cap, var=1):
        """Device-resident call: pointers are device addresses (ints); metas are
        (deg_x, deg_y, limbs); out_cap = (deg_cap, limbs_cap).  Asynchronous."""
        fb = _Bipoly(f_meta[0], f_meta[1], f_meta[2], f_ptr)
        gb = _Bipoly(g_meta[0], g_meta[1], g_meta[2], g_ptr)
        ob = _Upoly(out_cap[0], out_cap[1], out_ptr)
        self._check(self.lib.bs_resultant_device(self.h, C.byref(fb), C.byref(gb), int(var),
                                                 C.byref(ob)))

    def alu_probe(self, kind):
        v = C.c_double()
        self._check(self.lib.bs_alu_probe(self.h, int(kind), C.byref(v)))
        return v.value

    def profile(self, enable=True):
        self._check(self.lib.bs_profile(self.h, 1 if enable else 0))

    def stage_times(self):
        ms = np.zeros(5, dtype=np.float32)
        self._check(self.lib.bs_stage_times(self.h, ms.ctypes.data, 5))
        return [float(x) for x in ms]

    def device_status(self):
        self._check(self.lib.bs_device_status(self.h))

    # -- univariate -----------------------------------------------------------------
    def uni_resultant_modp(self, primes, a, b):
        """Resultants mod p of equal-shape univariate images: a[i], b[i] ascending lists."""
        n = len(primes)
        da = len(a[0]) - 1
        db = len(b[0]) - 1
        A = np.ascontiguousarray(np.array(a, dtype=np.uint32).reshape(n, da + 1))
        B = np.ascontiguousarray(np.array(b, dtype=np.uint32).reshape(n, db + 1))
        Pm = np.ascontiguousarray(np.array(primes, dtype=np.uint32))
        R = np.zeros(n, dtype=np.uint32)
        self._check(self.lib.bs_uni_resultant_modp(self.h, n, Pm.ctypes.data, A.ctypes.data, da,
                                                   da + 1, B.ctypes.data, db, db + 1,
                                                   R.ctypes.data))
        return [int(x) for x in R]

    def gcd_modp(self, a, b, p):
        """Monic gcd in Z_p[x] of ascending coefficient lists (values in [0, p))."""
        da, db = len(a) - 1, len(b) - 1
        A = np.ascontiguousarray(np.array(a if a else [0], dtype=np.uint32))
        B = np.ascontiguousarray(np.array(b if b else [0], dtype=np.uint32))
        G = np.zeros(max(da, db, 0) + 1, dtype=np.uint32)
        dg = C.c_int()
        self._check(self.lib.bs_gcd_modp(self.h, A.ctypes.data, da, B.ctypes.data, db,
                                         C.c_uint32(p), G.ctypes.data, C.byref(dg)))
        return [int(x) for x in G[: dg.value + 1]]

    def gcd_z(self, a, b):
        """gcd in Z[x] of ascending integer coefficient lists (positive leading coefficient)."""
        return self.modgcd_batch([(0, a, b)])[0]

    def modgcd_batch(self, jobs):
        """jobs: list of (kind, a, b); kind 0 gcd(a, b), kind 1 square-free part of a (b
        unused), kind 2 the exact quotient a / b (b must divide a in Z[x])."""
        n = len(jobs)
        kinds = (C.c_int * n)(*[int(k) for k, _, _ in jobs])
        keep = []
        A = (_Upoly * n)()
        Bv = (_Upoly * n)()
        for j, (k, a, b) in enumerate(jobs):
            for arr_list, poly in ((A, a), (Bv, b if k != 1 else [])):
                arr, L = ints_to_limbs(poly)
                keep.append(arr)
                arr_list[j] = _Upoly(len(poly) - 1, L, arr.ctypes.data)
        out = (_Upoly * n)()
        for j in range(n):
            out[j] = _Upoly(0, 0, None)
        self._check(self.lib.bs_modgcd_batch(self.h, n, C.cast(kinds, C.c_void_p),
                                             C.cast(A, C.c_void_p), C.cast(Bv, C.c_void_p),
                                             C.cast(out, C.c_void_p)))
        bufs = []
        for j in range(n):
            buf = np.zeros((max(out[j].deg, 0) + 1) * max(out[j].limbs, 1), dtype=np.uint32)
            bufs.append(buf)
            out[j] = _Upoly(out[j].deg, max(out[j].limbs, 1), buf.ctypes.data)
        self._check(self.lib.bs_modgcd_batch(self.h, n, C.cast(kinds, C.c_void_p),
                                             C.cast(A, C.c_void_p), C.cast(Bv, C.c_void_p),
                                             C.cast(out, C.c_void_p)))
        return [limbs_to_ints(bufs[j], out[j].deg + 1, out[j].limbs) if out[j].deg >= 0 else []
                for j in range(n)]

    def squarefree_factorization(self, r):
        """Yun's square-free factorisation of the ascending integer list r: the list
        [r_1, ..., r_s] of primitive factors (positive leading coefficients) with
        r = c * prod r_i**i; a constant has no factors."""
        return self.squarefree_factorization_batch([r])[0]

    def squarefree_factorization_batch(self, polys):
        n = len(polys)
        keep = []
        inp = (_Upoly * n)()
        for j, r in enumerate(polys):
            arr, L = ints_to_limbs(r)
            keep.append(arr)
            inp[j] = _Upoly(len(r) - 1, L, arr.ctypes.data)
        out = (_Upoly * n)()
        for j in range(n):
            out[j] = _Upoly(0, 0, None)
        nfac = np.zeros(n, dtype=np.int32)
        args = lambda cap, fdeg: (self.h, n, C.cast(inp, C.c_void_p), int(cap),
                                  fdeg.ctypes.data, nfac.ctypes.data, C.cast(out, C.c_void_p))
        fdeg = np.zeros(1, dtype=np.int32)
        self._check(self.lib.bs_squarefree_factorization_batch(*args(0, fdeg)))
        cap = max(1, int(nfac.max()) if n else 1)
        fdeg = np.zeros(n * cap, dtype=np.int32)
        bufs = []
        for j in range(n):
            buf = np.zeros((max(out[j].deg, 0) + 1) * max(out[j].limbs, 1), dtype=np.uint32)
            bufs.append(buf)
            out[j] = _Upoly(out[j].deg, max(out[j].limbs, 1), buf.ctypes.data)
        self._check(self.lib.bs_squarefree_factorization_batch(*args(cap, fdeg)))
        res = []
        for j in range(n):
            coefs = limbs_to_ints(bufs[j], out[j].deg + 1, out[j].limbs) if out[j].deg >= 0 else []
            facs, pos = [], 0
            for d in fdeg[j * cap: j * cap + int(nfac[j])]:
                facs.append(coefs[pos: pos + int(d) + 1])
                pos += int(d) + 1
            res.append(facs)
        return res

    # ---- serving loop -----------------------------------------------------------------
    def serve_start(self, slots=3, max_batch=64, arena_bytes=0):
        self._check(self.lib.bs_serve_start(self.h, int(slots), int(max_batch), int(arena_bytes)))
        self._serve_keep = {}

    def serve_stop(self):
        self._check(self.lib.bs_serve_stop(self.h))
        self._serve_keep = {}

    def submit(self, kind, *operands, var=1):
        """Queue a job: submit(JOB_RESULTANT, f, g, var=1), submit(JOB_GCD, a, b) or
        submit(JOB_SQFREE, a).  Returns the ticket."""
        job = _Job()
        job.kind = int(kind)
        job.var = int(var)
        keep = []
        if kind == JOB_RESULTANT:
            for name, poly in zip(("f", "g"), operands):
                arr, dx, dy, L = bipoly_to_limbs(poly)
                keep.append(arr)
                setattr(job, name, _bip(arr, dx, dy, L))
        else:
            polys = list(operands) + [[]] * (2 - len(operands))
            for name, poly in zip(("a", "b"), polys):
                arr, L = ints_to_limbs(poly)
                keep.append(arr)
                setattr(job, name, _Upoly(len(poly) - 1, L, arr.ctypes.data))
        t = C.c_uint64()
        self._check(self.lib.bs_submit(self.h, C.byref(job), C.byref(t)))
        return int(t.value)

    def poll(self, ticket):
        """None while the job runs; otherwise (status, coefficients, queue_ms, latency_ms)."""
        r = _Result()
        rc = self.lib.bs_poll(self.h, C.c_uint64(ticket), C.byref(r))
        if rc == BS_PENDING:
            return None
        self._check(rc)
        words = (r.deg + 1) * r.limbs
        buf = np.zeros(max(words, 1), dtype=np.uint32)
        r.c = buf.ctypes.data
        r.cap_words = buf.size
        self._check(self.lib.bs_poll(self.h, C.c_uint64(ticket), C.byref(r)))
        coeffs = limbs_to_ints(buf, r.deg + 1, r.limbs) if r.deg >= 0 else []
        return int(r.status), coeffs, float(r.queue_ms), float(r.latency_ms)

    def wait(self, ticket, timeout_ms=-1):
        rc = self.lib.bs_wait(self.h, C.c_uint64(ticket), int(timeout_ms))
        if rc == 4:
            return False
        self._check(rc)
        return True

    def serve_stats(self):
        info = _ServeInfo()
        self._check(self.lib.bs_serve_stats(self.h, C.byref(info)))
        return {name: getattr(info, name) for name, _ in _ServeInfo._fields_}

    def autotune_batch(self, pairs, var=1):
        """Tune the batched launch shapes on these pairs; returns the chosen shapes."""
        n = len(pairs)
        F, G, keep = (_Bipoly * n)(), (_Bipoly * n)(), []
        for i, (f, g) in enumerate(pairs):
            af, dxf, dyf, Lf = bipoly_to_limbs(f)
            ag, dxg, dyg, Lg = bipoly_to_limbs(g)
            keep += [af, ag]
            F[i] = _bip(af, dxf, dyf, Lf)
            G[i] = _bip(ag, dxg, dyg, Lg)
        info = _TuneInfo()
        self._check(self.lib.bs_autotune_batch(self.h, n, F, G, int(var), C.byref(info)))
        out = {name: getattr(info, name) for name, _ in _TuneInfo._fields_}
        out["uni_threads"] = list(info.uni_threads)
        return out

    def set_tune(self, eval_warps=8, eval_blocks_per_sm=5, uni_threads=(128,) * 6, crt_tile=8,
                 crt_blocks_per_sm=4, eval_independent=1):
        t = _TuneInfo()
        t.eval_warps, t.eval_blocks_per_sm = eval_warps, eval_blocks_per_sm
        for c in range(6):
            t.uni_threads[c] = uni_threads[c]
        t.crt_tile, t.crt_blocks_per_sm = crt_tile, crt_blocks_per_sm
        t.eval_independent = eval_independent
        self._check(self.lib.bs_set_tune(self.h, C.byref(t)))

    def squarefree_part(self, r):
        arr, L = ints_to_limbs(r)
        inp = _Upoly(len(r) - 1, L, arr.ctypes.data)
        out = _Upoly(0, 0, None)
        self._check(self.lib.bs_squarefree_part(self.h, C.byref(inp), C.byref(out)))
        buf = np.zeros((max(out.deg, 0) + 1) * out.limbs, dtype=np.uint32)
        out = _Upoly(out.deg, out.limbs, buf.ctypes.data)
        self._check(self.lib.bs_squarefree_part(self.h, C.byref(inp), C.byref(out)))
        return limbs_to_ints(buf, out.deg + 1, out.limbs) if out.deg >= 0 else []


# module-level functions with the C names -------------------------------------------

def bs_prime_table(count):
    lib = load_library()
    out = np.zeros(count, dtype=np.uint32)
    rc = lib.bs_prime_table(int(count), out.ctypes.data)
    if rc:
        raise BsError(rc, lib.bs_error_string(rc).decode())
    return [int(x) for x in out]


def bs_plan(f, g, var=1):
    """Host-only plan of res(f, g; var) as a dict (no GPU needed)."""
    lib = load_library()
    af, dxf, dyf, Lf = bipoly_to_limbs(f)
    ag, dxg, dyg, Lg = bipoly_to_limbs(g)
    fb, gb = _bip(af, dxf, dyf, Lf), _bip(ag, dxg, dyg, Lg)
    info = _PlanInfo()
    rc = lib.bs_plan(C.byref(fb), C.byref(gb), int(var), C.byref(info))
    if rc:
        raise BsError(rc, lib.bs_error_string(rc).decode())
    return {k: getattr(info, k) for k, _ in _PlanInfo._fields_}


def bs_resultant(ctx, f, g, var=1):
    return ctx.resultant(f, g, var)


def bs_resultant_batch(ctx, pairs, var=1):
    return ctx.resultant_batch(pairs, var)


def bs_resultant_bounds(ctx, f_meta, g_meta, var=1):
    return ctx.resultant_bounds(f_meta, g_meta, var)


def bs_resultant_device(ctx, *args, **kw):
    return ctx.resultant_device(*args, **kw)


def bs_device_status(ctx):
    return ctx.device_status()


def bs_uni_resultant_modp(ctx, primes, a, b):
    return ctx.uni_resultant_modp(primes, a, b)


def bs_gcd_modp(ctx, a, b, p):
    return ctx.gcd_modp(a, b, p)


def bs_squarefree_part(ctx, r):
    return ctx.squarefree_part(r)
