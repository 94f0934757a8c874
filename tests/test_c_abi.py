"""The boundary is a C ABI: include/subcull.h compiles as C11 with
-pedantic and no warnings, and a C program links against libsubcull.so and
calls it (build options, the ray-mask tables and a host-side build; no
device calls)."""
import os
import shutil
import subprocess

import pytest

from paper_2305_08343_gb300 import _build

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include "subcull.h"
#include <stdio.h>
#include <stdlib.h>

int main(void) {
  if (sc_abi_version() != SC_ABI_VERSION || SC_ABI_VERSION != 2) return 1;
  sc_build_opts o;
  sc_build_opts_default(&o);
  if (o.max_leaf != 4 || o.bins != 32 || o.gpu_bvh != 0 || o.gpu_masks != 0) return 2;
  uint32_t* lut = (uint32_t*)malloc(sizeof(uint32_t) * 64 * 64 * 2);
  if (sc_raylut(4, lut) != SC_OK) return 3;
  /* one triangle: a leaf root, no inner node */
  const float tri[9] = {0, 0, 0, 1, 0, 0, 0, 1, 0};
  sc_bvh* b = NULL;
  if (sc_bvh_build(tri, 1, 4, 0, &o, &b) != SC_OK || !b) return 4;
  sc_bvh_info info;
  if (sc_bvh_get_info(b, &info) != SC_OK || info.num_tris != 1 || info.num_nodes != 0) return 5;
  sc_refit_info r;
  if (sc_bvh_refit(b, tri, 1, &r) != SC_OK || r.moved_tris != 0) return 6;
  sc_bvh* bad = NULL;
  if (sc_bvh_build(tri, 1, 5, 0, &o, &bad) != SC_ERR_UNSUPPORTED || bad) return 7;
  if (sc_last_error()[0] == 0) return 8;
  sc_bvh_destroy(b);
  free(lut);
  printf("c abi ok\n");
  return 0;
}
"""


def test_header_is_c_and_a_c_program_links(tmp_path):
    if shutil.which("gcc") is None:
        pytest.skip("gcc not available")
    so = _build.build_product()
    src = tmp_path / "abi.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "abi"
    cmd = ["gcc", "-std=c11", "-Wall", "-Wextra", "-pedantic", "-Werror",
           "-I" + os.path.join(ROOT, "include"), str(src), "-o", str(exe),
           so, "-Wl,-rpath," + os.path.dirname(so)]
    r = subprocess.run(cmd, capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0 and "c abi ok" in out.stdout, (out.returncode, out.stderr)
