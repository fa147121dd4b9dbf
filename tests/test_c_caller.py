"""The C ABI from a plain C program: include/sfx.h compiles as ISO C99 with
-pedantic, and a C caller linked against libsfx.so gets the 1D Gauss rule and
Lagrange tables (host-side entry points, no GPU) and the documented status for
bad arguments.  The rule is checked against numpy's Gauss-Legendre nodes and
weights, mapped to [0, 1] (Sec. 1.2, Eq. tpps)."""
import os
import shutil
import subprocess

import numpy as np
import pytest

import paper_1711_02473_gb300 as sfx

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include "sfx.h"

int main(void) {
  double x[9], w[9], t[81];
  /* 9 Gauss points, Lagrange basis on 9 GLL nodes, values then derivatives */
  sfx_status s = sfx_tabulate_1d(SFX_NODES_GLL, 9, SFX_NODES_GL, 9, 0, x, w, t);
  if (s != SFX_OK) return 1;
  for (int i = 0; i < 9; ++i) printf("%.17g %.17g\n", x[i], w[i]);
  double rowsum = 0.0;
  for (int q = 0; q < 9; ++q)
    for (int i = 0; i < 9; ++i) rowsum += t[q * 9 + i];
  printf("%.17g\n", rowsum);
  s = sfx_tabulate_1d(SFX_NODES_GLL, 9, SFX_NODES_GL, 9, 1, NULL, NULL, t);
  if (s != SFX_OK) return 2;
  double dsum = 0.0;
  for (int k = 0; k < 81; ++k) dsum += t[k];
  printf("%.17g\n", dsum);
  /* nq = 0 is an argument error */
  s = sfx_tabulate_1d(SFX_NODES_GLL, 9, SFX_NODES_GL, 0, 0, x, w, t);
  printf("%d %s\n", (int)s, sfx_status_string(s));
  return 0;
}
"""


@pytest.fixture(scope="module")
def libdir():
    sfx.build()
    return os.path.dirname(sfx.LIB_PATH)


def test_header_is_iso_c99(tmp_path):
    src = tmp_path / "h.c"
    src.write_text('#include "sfx.h"\nint main(void) { return (int)sizeof(sfx_form_params) == 0; }\n')
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only",
                        "-I", os.path.join(ROOT, "include"), str(src)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr


@pytest.mark.skipif(shutil.which("gcc") is None, reason="no C compiler")
def test_c_program_calls_the_library(tmp_path, libdir):
    src = tmp_path / "caller.c"
    exe = tmp_path / "caller"
    src.write_text(PROGRAM)
    r = subprocess.run(["gcc", "-std=c99", "-Wall", "-Werror", "-I", os.path.join(ROOT, "include"), str(src),
                        "-o", str(exe), "-L", libdir, "-lsfx", "-Wl,-rpath," + libdir], capture_output=True,
                       text=True)
    assert r.returncode == 0, r.stderr
    r = subprocess.run([str(exe)], capture_output=True, text=True, timeout=60)
    assert r.returncode == 0, (r.returncode, r.stderr)
    lines = r.stdout.split("\n")
    xw = np.array([[float(v) for v in lines[i].split()] for i in range(9)])
    t, wt = np.polynomial.legendre.leggauss(9)
    order = np.argsort(xw[:, 0])
    np.testing.assert_allclose(xw[order, 0], 0.5 * (t + 1.0), rtol=0, atol=1e-15)
    np.testing.assert_allclose(xw[order, 1], 0.5 * wt, rtol=0, atol=1e-15)
    assert abs(float(lines[9]) - 9.0) < 1e-13     # each row of the value table sums to 1
    assert abs(float(lines[10])) < 1e-11          # each row of the derivative table sums to 0
    code, msg = lines[11].split(" ", 1)
    assert int(code) == -1 and msg.strip()         # SFX_ERR_ARG with its message
