"""The boundary is a C ABI: a plain C99 program includes include/bsres.h, links against
libbsres.so and calls the host-only entry points (prime table, planner, size bounds, error
strings); its answers must agree with the Python binding and with the oracle's plan."""

import os
import shutil
import subprocess

import pytest

import paper_1201_1548_gb300 as bs
from oracle import numtheory as nt
from oracle import resultant as R

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))
PKG = os.path.join(ROOT, "paper_1201_1548_gb300")

SOURCE = r"""
#include <stdio.h>
#include "bsres.h"

int main(void) {
  uint32_t pr[4];
  /* f = x^2 + y^2 - 1 on a 3 x 3 grid, g = y - x on a 2 x 2 grid (one limb each) */
  const uint32_t fc[9] = {0xffffffffu, 0u, 1u, 0u, 0u, 0u, 1u, 0u, 0u};
  const uint32_t gc[4] = {0u, 0xffffffffu, 1u, 0u};
  bs_bipoly f, g;
  bs_plan_info pi;
  int32_t d = 0, L = 0;
  f.deg_x = 2; f.deg_y = 2; f.limbs = 1; f.c = fc;
  g.deg_x = 1; g.deg_y = 1; g.limbs = 1; g.c = gc;
  if (bs_prime_table(4, pr) != BS_OK) return 1;
  printf("%u %u %u %u\n", pr[0], pr[1], pr[2], pr[3]);
  if (bs_plan(&f, &g, 1, &pi) != BS_OK) return 2;
  printf("%d %d %d %d %d %d %d %d\n", pi.trivial, pi.m_e, pi.n_e, pi.D, pi.N, pi.k_need, pi.k_total,
         pi.out_limbs);
  if (bs_resultant_bounds(&f, &g, 1, &d, &L) != BS_OK) return 3;
  printf("%d %d\n", d, L);
  printf("%s\n", bs_error_string(BS_ERR_ZERO));
  return 0;
}
"""


def test_c_program_uses_the_library(tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    from paper_1201_1548_gb300.build import build
    build()
    src = tmp_path / "consumer.c"
    src.write_text(SOURCE)
    exe = tmp_path / "consumer"
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-I", os.path.join(ROOT, "include"),
                    str(src), "-o", str(exe), "-L", PKG, "-lbsres", "-Wl,-rpath," + PKG], check=True)
    lines = subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines()

    assert [int(v) for v in lines[0].split()] == nt.prime_table(4)
    trivial, m_e, n_e, D, N, k_need, k_total, out_limbs = (int(v) for v in lines[1].split())
    f = [[-1, 0, 1], [0, 0, 0], [1, 0, 0]]
    g = [[0, -1], [1, 0]]
    ours = bs.bs_plan(f, g, 1)
    assert (trivial, m_e, n_e, D, N, k_need, k_total, out_limbs) == (
        ours["trivial"], ours["m_e"], ours["n_e"], ours["D"], ours["N"], ours["k_need"], ours["k_total"],
        ours["out_limbs"])
    ref = R.plan(f, g, 1, nt.prime_table(50))
    assert (m_e, n_e, D, N) == (ref["m_y"], ref["n_y"], ref["D"], ref["N"]) == (2, 1, 2, 4)
    assert ref["k"] <= k_need <= ref["k"] + 1
    d, L = (int(v) for v in lines[2].split())
    assert d >= D and L >= out_limbs
    assert lines[3] == bs.load_library().bs_error_string(bs.BS_ERR_ZERO).decode()
