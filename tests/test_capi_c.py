"""The boundary is a C ABI: include/pepsi.h compiles as C99, and a plain C
program links the library and calls its host-only functions (parameter
selection, error strings) without a GPU."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_PROGRAM = r"""
#include "pepsi.h"
#include <stdio.h>
#include <string.h>
int main(void) {
  double bits = 0; uint64_t ell = 0; uint32_t ln = 0, lq = 0, h = 0;
  if (pepsi_request_bits(19, 8, 8192, &bits, &ell, &ln, &lq) != PEPSI_OK) return 1;
  if (ell != 24 || ln != 13 || lq != 204) return 2;            /* Eq. 1 and Table 3 */
  if (pepsi_comm_optimal_h(48, 4096, 64, &h) != PEPSI_OK || h != 23) return 3;  /* Section 6.1 */
  if (pepsi_request_bits(19, 0, 8192, &bits, 0, 0, 0) != PEPSI_E_PARAM) return 4;
  if (strlen(pepsi_strerror(PEPSI_E_NOISE)) == 0) return 5;
  puts("ok");
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib_path():
    from paper_2310_14565_gb300 import build

    return build.build()


def test_header_is_c99():
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    subprocess.run(["gcc", "-std=c99", "-Wall", "-Wextra", "-pedantic", "-Werror", "-fsyntax-only", "-x", "c",
                    os.path.join(ROOT, "include", "pepsi.h")], check=True)


def test_c_program_calls_the_library(lib_path, tmp_path):
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    src = tmp_path / "prog.c"
    src.write_text(C_PROGRAM)
    exe = tmp_path / "prog"
    libdir = os.path.dirname(lib_path)
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-L", libdir,
                    "-lpepsi_gb300", "-Wl,-rpath," + libdir, "-o", str(exe)], check=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and out.stdout.strip() == "ok", (out.returncode, out.stdout, out.stderr)
