"""libswkb.so used from plain C, the way a non-Python caller would: a C
program built with gcc against include/swkb.h reads a problem (permittivity
table, domain, options, incident field) from a binary file, propagates it
through the C ABI (host buffers), and writes the field; it must equal the
Python binding's result for the same problem bit for bit."""
import os
import shutil
import subprocess

import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

C_SOURCE = r"""
#include <stdio.h>
#include <stdlib.h>
#include "swkb.h"

/* problem file: int32 n_p, n_z, bc, precision, ray_stride, rk4_steps, n_screens,
   fc_patch, fc_overlap;
   double z0_p, dz_p, k, z_a, z_b, dx, theta_max;
   double eps[n_p], eps_z[n_p], eps_zz[n_p]; double u0[2 n_z] */
int main(int argc, char** argv) {
  if (argc != 3) return 2;
  FILE* f = fopen(argv[1], "rb");
  if (!f) return 3;
  int32_t hdr[9];
  double d[7];
  if (fread(hdr, sizeof(int32_t), 9, f) != 9 || fread(d, sizeof(double), 7, f) != 7) return 4;
  const int n_p = hdr[0], n_z = hdr[1];
  double* tab = malloc(sizeof(double) * 3 * (size_t)n_p);
  double* u0 = malloc(sizeof(double) * 2 * (size_t)n_z);
  double* out = malloc(sizeof(double) * 2 * (size_t)n_z);
  if (fread(tab, sizeof(double), 3 * (size_t)n_p, f) != 3 * (size_t)n_p) return 5;
  if (fread(u0, sizeof(double), 2 * (size_t)n_z, f) != 2 * (size_t)n_z) return 6;
  fclose(f);
  const double x_col = 0.0;
  swkb_profile prof = {1, &x_col, n_p, d[0], d[1], tab, tab + n_p, tab + 2 * (size_t)n_p};
  swkb_domain dom = {d[3], d[4], 0.0, hdr[2]};
  swkb_options opt;
  swkb_options_default(&opt);
  opt.precision = hdr[3];
  opt.ray_stride = hdr[4];
  opt.rk4_steps = hdr[5];
  opt.theta_max = d[6];
  opt.fc_patch = hdr[7];
  opt.fc_overlap = hdr[8];
  swkb_plan* plan = NULL;
  swkb_status st = swkb_plan_create(&prof, d[2], &dom, n_z, d[5], &opt, &plan);
  if (st != SWKB_OK) { fprintf(stderr, "create: %s\n", swkb_last_error()); return 10 + st; }
  swkb_plan_info info;
  swkb_plan_get_info(plan, &info);
  st = swkb_propagate(plan, u0, 0, hdr[6], out, 0, 0);
  if (st != SWKB_OK) { fprintf(stderr, "propagate: %s\n", swkb_last_error()); return 30 + st; }
  swkb_plan_destroy(plan);
  f = fopen(argv[2], "wb");
  fwrite(out, sizeof(double), 2 * (size_t)n_z, f);
  fclose(f);
  printf("modes %d rays %d\n", info.n_modes, info.n_rays_total);
  free(tab); free(u0); free(out);
  return 0;
}
"""


PROBLEMS = {
    "grounded-duct": lambda: w.config_surface_duct_small(n_screens=3).with_(absorber_frac=0.0),
    "open-lens": lambda: w.config_open_lens(n_z=1000, fc_patch=280, fc_overlap=100,
                                            n_screens=2),
}


@pytest.mark.parametrize("name", sorted(PROBLEMS))
@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_c_program_matches_the_binding(tmp_path, prec, name):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    cc = shutil.which("gcc") or shutil.which("cc")
    if cc is None:
        pytest.skip("no C compiler")
    pb = PROBLEMS[name]()
    pr = pb.profile
    src = tmp_path / "client.c"
    src.write_text(C_SOURCE)
    exe = tmp_path / "client"
    libdir = os.path.dirname(swkb.LIB_PATH)
    subprocess.run([cc, "-std=c11", "-O2", "-I", os.path.join(ROOT, "include"), str(src), "-o",
                    str(exe), "-L", libdir, "-lswkb", f"-Wl,-rpath,{libdir}"], check=True,
                   capture_output=True)
    blob = tmp_path / "problem.bin"
    with open(blob, "wb") as f:
        np.array([pr.n_p, pb.n_z, pb.bc, prec, pb.ray_stride, pb.rk4_steps, pb.n_screens,
                  pb.fc_patch, pb.fc_overlap], np.int32).tofile(f)
        np.array([pr.z0, pr.dz, pb.k, pb.z_a, pb.z_b, pb.dx, pb.theta_max], np.float64).tofile(f)
        np.concatenate([pr.eps[0], pr.eps_z[0], pr.eps_zz[0]]).astype(np.float64).tofile(f)
        np.ascontiguousarray(pb.u0, np.complex128).view(np.float64).tofile(f)
    out = tmp_path / "field.bin"
    r = subprocess.run([str(exe), str(blob), str(out)], capture_output=True, text=True)
    assert r.returncode == 0, r.stderr
    got = np.fromfile(out, np.float64).view(np.complex128)
    want = swkb.Plan(pb, prec).propagate()
    assert np.array_equal(got, want)
