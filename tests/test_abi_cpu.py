"""CPU-side checks of the C ABI: the library loads, exports every declared symbol, and its
host-only parts (prime table, planner, size bounds) agree with the oracle."""

import os
import re

import numpy as np
import pytest

import paper_1201_1548_gb300 as bs
from oracle import numtheory as nt
from oracle import resultant as R
from workloads import cfg1_pair, cfg2_pair, cfg3_batch, dense_curve

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))


@pytest.fixture(scope="module", autouse=True)
def built():
    from paper_1201_1548_gb300.build import build
    build()


def _declared_symbols():
    text = open(os.path.join(ROOT, "include", "bsres.h")).read()
    text = re.sub(r"/\*.*?\*/", "", text, flags=re.S)
    return sorted(set(re.findall(r"\b(bs_[a-z_0-9]+)\s*\(", text)))


def test_every_declared_symbol_is_exported():
    lib = bs.load_library()
    declared = _declared_symbols()
    assert len(declared) >= 14
    for name in declared:
        assert hasattr(lib, name), name
    assert sorted(bs.EXPORTED_SYMBOLS) == declared


def test_debug_build_exports_the_same_entry_points():
    """The debug build (kernels bounds-check their accesses, BS_DEBUG_CHECKS) compiles,
    links and exports every declared entry point."""
    import ctypes
    from paper_1201_1548_gb300.build import build
    path = build(debug=True)
    assert path.endswith("libbsres_debug.so")
    lib = ctypes.CDLL(path)
    for name in _declared_symbols():
        assert hasattr(lib, name), name


def test_prime_table_matches_oracle_definition():
    ours = bs.bs_prime_table(300)
    assert ours == nt.prime_table(300)


def test_marshalling_roundtrip():
    vals = [0, 1, -1, 2**31 - 1, -2**31, 2**63, -(2**200) + 12345, 3**100]
    arr, L = bs.ints_to_limbs(vals)
    assert bs.limbs_to_ints(arr, len(vals), L) == vals
    arr2, L2 = bs.ints_to_limbs([5, -5], limbs=3)
    assert L2 == 3 and bs.limbs_to_ints(arr2, 2, 3) == [5, -5]


def _oracle_k(f, g, var):
    primes = nt.prime_table(2000)
    return R.plan(f, g, var, primes)


def _lead_row(f, var):
    """Coefficients of the leading row in the eliminated variable (var 1: y)."""
    grid = [list(r) for r in f]
    if var == 0:  # rows by powers of x
        width = max(len(r) for r in grid)
        grid = [[grid[j][i] if i < len(grid[j]) else 0 for j in range(len(grid))]
                for i in range(width)]
    for row in reversed(grid):
        if any(row):
            return row
    return []


def _check_spares(f, g, var, plan):
    """Spare primes: the smallest K such that [0, K) holds k_need primes (plus two when a
    leading row is not a monomial) dividing neither leading row's smallest coefficient."""
    rows = [_lead_row(f, var), _lead_row(g, var)]
    mins = []
    for row in rows:
        nz = [(abs(c).bit_length(), o, c) for o, c in enumerate(row) if c]
        mins.append(min(nz)[2])
    coset = 0 if all(sum(1 for c in row if c) == 1 for row in rows) else 2
    want = plan["k_need"] + coset
    K = plan["k_total"]
    primes = nt.prime_table(K)
    div = [any(c % p == 0 for c in mins) for p in primes]
    assert K - sum(div) >= want
    assert K == want or (K - 1) - sum(div[:-1]) < want      # the smallest such K
    # every prime that rejects the job (dividing a whole leading row) is among them
    for p, dv in zip(primes, div):
        if any(all(c % p == 0 for c in row) for row in rows):
            assert dv


@pytest.mark.parametrize("var", [1, 0])
def test_planner_matches_oracle(var):
    cases = [cfg1_pair(1), cfg1_pair(2), cfg2_pair(1)]
    rng = np.random.Generator(np.random.PCG64(5))
    for _ in range(6):
        cases.append((dense_curve(rng, int(rng.integers(1, 9)), int(rng.integers(2, 300))),
                      dense_curve(rng, int(rng.integers(1, 9)), int(rng.integers(2, 300)))))
    cases += cfg3_batch(seed=3, count=8)
    for f, g in cases:
        ours = bs.bs_plan(f, g, var)
        ref = _oracle_k(f, g, var)
        assert ours["m_e"] == ref["m_y"] and ours["n_e"] == ref["n_y"]
        assert ours["D"] == ref["D"]
        assert ours["N"] == ref["N"]
        # the planner's bound is an upper bound within one bit of the exact one
        assert ref["k"] <= ours["k_need"] <= ref["k"] + 1
        _check_spares(f, g, var, ours)
        # output limbs hold the bound
        assert 32 * ours["out_limbs"] >= (ref["bound_sq"].bit_length() + 1) // 2 + 1


def test_planner_trivial_cases():
    zero = [[0, 0], [0, 0]]
    g = [[1, 2], [3, 0]]
    assert bs.bs_plan(zero, g, 1)["trivial"] == 1
    assert bs.bs_plan([[5]], [[7, 1]], 1)["trivial"] == 2   # both constant in y
    p = bs.bs_plan([[1, 1], [2, 0]], [[3, 1]], 1)           # g constant in y: R = g^{m}
    assert p["trivial"] == 0 and p["m_e"] == 1 and p["n_e"] == 0


def test_resultant_bounds_cover_plans():
    lib = bs.load_library()
    import ctypes as C
    for f, g in [cfg1_pair(1), cfg2_pair(1)] + cfg3_batch(seed=4, count=6):
        af, dxf, dyf, Lf = bs.bipoly_to_limbs(f)
        ag, dxg, dyg, Lg = bs.bipoly_to_limbs(g)
        from paper_1201_1548_gb300._abi import _Bipoly
        fb, gb = _Bipoly(dxf, dyf, Lf, None), _Bipoly(dxg, dyg, Lg, None)
        d, L = C.c_int32(), C.c_int32()
        assert lib.bs_resultant_bounds(C.byref(fb), C.byref(gb), 1, C.byref(d), C.byref(L)) == 0
        p = bs.bs_plan(f, g, 1)
        assert d.value >= p["D"] and L.value >= p["out_limbs"]


def test_no_cpu_fallback_without_a_gpu():
    # every compute entry point needs a context, and a context needs a CUDA device: on a
    # machine without one the library reports a CUDA error instead of computing on the host
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    with pytest.raises(bs.BsError) as e:
        bs.Context(0)
    assert e.value.code == bs.BS_ERR_CUDA


def test_missing_library_raises(monkeypatch, tmp_path):
    from paper_1201_1548_gb300 import _abi
    monkeypatch.setattr(_abi, "_LIB", None)
    monkeypatch.setattr(_abi, "_LIB_PATH", str(tmp_path / "libbsres.so"))
    with pytest.raises(bs.BsError):
        _abi.load_library()


def test_planner_rejects_malformed_inputs():
    import ctypes as C
    from paper_1201_1548_gb300._abi import _Bipoly, _PlanInfo
    lib = bs.load_library()
    buf = np.zeros(2 * 2 * 65, dtype=np.uint32)
    buf[0] = 1

    def plan(f, g, var=1):
        info = _PlanInfo()
        return lib.bs_plan(C.byref(f) if f is not None else None, C.byref(g), var, C.byref(info))

    ok = _Bipoly(1, 1, 1, buf.ctypes.data)
    assert plan(ok, ok) == bs.BS_OK
    assert plan(_Bipoly(1, 1, 64, buf.ctypes.data), ok) == bs.BS_OK       # the widest coefficients
    for bad in (_Bipoly(1, 1, 0, buf.ctypes.data), _Bipoly(1, 1, 65, buf.ctypes.data),
                _Bipoly(-1, 1, 1, buf.ctypes.data), _Bipoly(1, -1, 1, buf.ctypes.data),
                _Bipoly(1, 1, 1, None)):
        assert plan(bad, ok) == bs.BS_ERR_ARG
        assert plan(ok, bad) == bs.BS_ERR_ARG
    assert plan(None, ok) == bs.BS_ERR_ARG
    assert plan(ok, ok, 2) == bs.BS_ERR_ARG


def test_smoke_needs_the_gpu():
    # the smoke check compares the CUDA path with the oracle; without a GPU it must fail,
    # not pass on some other path
    torch = pytest.importorskip("torch")
    if torch.cuda.is_available():
        pytest.skip("a GPU is present")
    import __graft_entry__ as entry
    with pytest.raises(bs.BsError) as e:
        entry.smoke()
    assert e.value.code == bs.BS_ERR_CUDA
