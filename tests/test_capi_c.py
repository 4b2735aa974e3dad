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


LAYOUT_PROGRAM = r"""
#include "pepsi.h"
#include <stddef.h>
#include <stdio.h>
int main(void) {
  printf("pepsi_params %zu %zu %zu\n", sizeof(pepsi_params), offsetof(pepsi_params, gamma),
         offsetof(pepsi_params, client_cuckoo));
  printf("pepsi_info %zu %zu\n", sizeof(pepsi_info), offsetof(pepsi_info, gamma));
  printf("pepsi_schedule %zu %zu\n", sizeof(pepsi_schedule), offsetof(pepsi_schedule, batch_requests));
  printf("pepsi_lane %zu %zu\n", sizeof(pepsi_lane), offsetof(pepsi_lane, slots));
  printf("pepsi_engine_stats %zu %zu\n", sizeof(pepsi_engine_stats), offsetof(pepsi_engine_stats, budget));
  return 0;
}
"""


def test_binding_structs_match_the_header(tmp_path):
    """The ctypes mirrors of the header's structs have the C layout: size and
    the offset of a late field of each, as a C compiler lays them out."""
    if not shutil.which("gcc"):
        pytest.skip("no C compiler")
    import ctypes as C

    import paper_2310_14565_gb300 as pepsi

    src = tmp_path / "layout.c"
    src.write_text(LAYOUT_PROGRAM)
    exe = tmp_path / "layout"
    subprocess.run(["gcc", "-std=c99", "-Wall", "-I", os.path.join(ROOT, "include"), str(src), "-o", str(exe)],
                   check=True)
    got = {}
    for line in subprocess.run([str(exe)], capture_output=True, text=True, check=True).stdout.splitlines():
        name, *vals = line.split()
        got[name] = [int(v) for v in vals]
    want = {
        "pepsi_params": [C.sizeof(pepsi.Params), pepsi.Params.gamma.offset, pepsi.Params.client_cuckoo.offset],
        "pepsi_info": [C.sizeof(pepsi.Info), pepsi.Info.gamma.offset],
        "pepsi_schedule": [C.sizeof(pepsi.Schedule), pepsi.Schedule.batch_requests.offset],
        "pepsi_lane": [C.sizeof(pepsi.LaneDesc), pepsi.LaneDesc.slots.offset],
        "pepsi_engine_stats": [C.sizeof(pepsi.EngineStats), pepsi.EngineStats.budget.offset],
    }
    assert got == want
