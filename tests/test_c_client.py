"""The C ABI from a plain C99 client: include/sc_lbm.h compiles as C with all
warnings as errors, the program links against the built library, and the calls
that need no GPU behave as the header states (direction table, tile list,
required bytes of both layouts, rejection of invalid parameters with a message)."""
import os
import shutil
import subprocess

import pytest

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

PROGRAM = r"""
#include <stdio.h>
#include <string.h>
#include "sc_lbm.h"

static sc_params base(void) {
  sc_params p;
  memset(&p, 0, sizeof p);
  p.nx = 64; p.ny = 64; p.nz = 64;
  p.tau_r = 1.0; p.tau_b = 1.0; p.G = 3.6; p.rho_H = 0.03;
  p.geometry = SC_GEOM_PLANAR_SINK; p.sink_z0 = 63; p.sink_layers = 1;
  p.storage = SC_STORAGE_F32; p.layout = SC_LAYOUT_TWO_LATTICE;
  return p;
}

int main(void) {
  int32_t c[19 * 3];
  double w[19], wsum = 0.0;
  if (sc_lattice_directions(c, w) != SC_OK) return 1;
  for (int i = 0; i < 19; ++i) wsum += w[i];
  if (wsum < 1.0 - 1e-12 || wsum > 1.0 + 1e-12) return 2;
  int32_t n = 0, tx[16], ty[16];
  if (sc_tile_list(&n, tx, ty, 16) != SC_OK || n < 1) return 3;
  sc_params p = base();
  size_t two = 0, aa = 0;
  if (sc_lbm_required_bytes(&p, &two) != SC_OK) return 4;
  p.layout = SC_LAYOUT_AA;
  if (sc_lbm_required_bytes(&p, &aa) != SC_OK) return 5;
  if (!(aa < two)) return 6;
  p = base();
  p.tau_r = 0.5;
  if (sc_lbm_required_bytes(&p, &two) != SC_EINVAL) return 7;
  if (strlen(sc_last_error()) == 0) return 8;
  p = base();
  p.G_rr = 1.0 / 0.0;
  if (sc_lbm_required_bytes(&p, &two) != SC_EINVAL) return 9;
  printf("%d tiles, two lattices %zu bytes, in place %zu bytes\n", (int)n, two, aa);
  return 0;
}
"""


@pytest.fixture(scope="module")
def lib():
    from paper_1701_03637_gb300 import _native
    _native.build()
    return _native.LIB_PATH


def test_c99_client_builds_links_and_runs(lib, tmp_path):
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    src = tmp_path / "client.c"
    src.write_text(PROGRAM)
    exe = tmp_path / "client"
    libdir = os.path.dirname(lib)
    libname = os.path.basename(lib)
    assert libname.startswith("lib") and libname.endswith(".so")
    subprocess.run([cc, "-std=c99", "-Wall", "-Wextra", "-Werror", "-pedantic", "-I", os.path.join(ROOT, "include"),
                    str(src), "-L", libdir, "-l" + libname[3:-3], "-Wl,-rpath," + libdir, "-o", str(exe)],
                   check=True, capture_output=True, text=True)
    out = subprocess.run([str(exe)], capture_output=True, text=True)
    assert out.returncode == 0, (out.returncode, out.stdout, out.stderr)
    assert "tiles" in out.stdout
