"""The 31-bit modular arithmetic of the kernels (Montgomery's reduction with predicate-free
corrections, modular add / subtract / negate, powers, Fermat inverses and Shoup's products
by a fixed factor) is compiled for
the host as well as the device; here its host build is checked against Python integers
on the extreme inputs its preconditions allow, for primes at both ends of the table."""

import os
import random
import shutil
import subprocess

import pytest

import paper_1201_1548_gb300 as bs

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
CSRC = os.path.join(ROOT, "paper_1201_1548_gb300", "csrc")

HARNESS = r"""
#include <cstdio>
#include <cinttypes>
#include "modarith.cuh"
using namespace bs;
int main() {
  unsigned op;
  uint64_t p, x, y;
  while (std::scanf("%u %" SCNu64 " %" SCNu64 " %" SCNu64, &op, &p, &x, &y) == 4) {
    const Mod M{(uint32_t)p, host_pinv((uint32_t)p)};
    const uint32_t one_m = host_to_mont(1, p);
    uint64_t r = 0;
    switch (op) {
      case 0: r = redc(x, M.p, M.pinv); break;
      case 1: r = redc_wide(x, M.p, M.pinv); break;
      case 2: r = mmul((uint32_t)x, (uint32_t)y, M); break;
      case 3: r = madd((uint32_t)x, (uint32_t)y, M.p); break;
      case 4: r = msub((uint32_t)x, (uint32_t)y, M.p); break;
      case 5: r = mneg((uint32_t)x, M.p); break;
      case 6: r = mpow((uint32_t)x, (uint32_t)y, one_m, M); break;
      case 7: r = minv((uint32_t)x, one_m, M); break;
      case 8: r = M.pinv; break;
      case 9: r = host_to_mont(x, p); break;
      case 10: r = host_powmod(x, y, p); break;
      case 11: r = mmul_shoup((uint32_t)x, (uint32_t)y, (uint32_t)((y << 32) / p), M.p); break;
    }
    std::printf("%" PRIu64 "\n", r);
  }
  return 0;
}
"""


@pytest.fixture(scope="module")
def harness(tmp_path_factory):
    cxx = shutil.which("g++")
    if cxx is None:
        pytest.skip("no host C++ compiler")
    d = tmp_path_factory.mktemp("modarith")
    src = d / "harness.cpp"
    src.write_text(HARNESS)
    exe = d / "harness"
    subprocess.run([cxx, "-std=c++17", "-O2", "-Wall", "-I", CSRC, str(src), "-o", str(exe)], check=True)

    def run(cases):
        text = "".join(f"{op} {p} {x} {y}\n" for op, p, x, y in cases)
        out = subprocess.run([str(exe)], input=text, capture_output=True, text=True, check=True).stdout
        return [int(v) for v in out.split()]

    return run


def _primes():
    table = bs.bs_prime_table(2000)
    return table[:3] + table[-3:]


def test_montgomery_reduction(harness):
    rng = random.Random(31)
    cases, want = [], []
    R = 1 << 32
    for p in _primes():
        rinv = pow(R, -1, p)
        # redc: t < p 2^32;  redc_wide: t < 2^32 * 1.5 p, as the kernels use it
        for t in [0, 1, p - 1, p, R - 1, R, p * R - 1, (p - 1) * R] + [rng.randrange(p * R) for _ in range(200)]:
            cases.append((0, p, t, 0))
            want.append(t * rinv % p)
        for t in [p * R, p * R + R - 1, 3 * p * R // 2 - 1] + [rng.randrange(3 * p * R // 2) for _ in range(200)]:
            cases.append((1, p, t, 0))
            want.append(t * rinv % p)
        # three products of values below p, the fused elimination step's sum
        for _ in range(100):
            t = sum(rng.randrange(p) * rng.randrange(p) for _ in range(3))
            cases.append((1, p, t, 0))
            want.append(t * rinv % p)
        cases.append((8, p, 0, 0))
        want.append(pow(p, -1, R))
    assert harness(cases) == want


def test_modular_operations(harness):
    rng = random.Random(32)
    cases, want = [], []
    R = 1 << 32
    for p in _primes():
        rinv = pow(R, -1, p)
        edge = [0, 1, 2, p - 2, p - 1]
        vals = edge + [rng.randrange(p) for _ in range(60)]
        for a in vals:
            b = rng.choice(vals)
            cases += [(2, p, a, b), (3, p, a, b), (4, p, a, b), (5, p, a, 0)]
            want += [a * b * rinv % p, (a + b) % p, (a - b) % p, (-a) % p]
        for a in edge + [rng.randrange(p) for _ in range(20)]:
            am = a * R % p                            # Montgomery form
            e = rng.choice([0, 1, 2, p - 2, p - 1, rng.randrange(1 << 32)])
            cases.append((6, p, am, e))
            want.append(pow(a, e, p) * R % p)
            if a:
                cases.append((7, p, am, 0))
                want.append(pow(a, -1, p) * R % p)
            cases.append((9, p, a, 0))
            want.append(am)
            cases.append((10, p, a, e))
            want.append(pow(a, e, p))
    assert harness(cases) == want


def test_shoup_products(harness):
    """x w mod p by Shoup's method (the transforms' short stages) for x, w below p, at the
    ends of both runs of the table (primes with 3p < 2^32 first, then up to 2^31)."""
    rng = random.Random(33)
    cases, want = [], []
    table = bs.bs_prime_table(6213)
    for p in table[:2] + table[2085:2089] + table[-2:]:
        edge = [0, 1, 2, p - 2, p - 1]
        for x in edge + [rng.randrange(p) for _ in range(100)]:
            for w in (rng.choice(edge), rng.randrange(p)):
                cases.append((11, p, x, w))
                want.append(x * w % p)
    assert harness(cases) == want
