"""The bounds-checked build (libswkb_checked.so, compiled with
-DSWKB_BOUNDS_CHECK) in place of a memory sanitizer: in the march, bracket
and resummation kernels every checked index is compared with its buffer, and
a violation is clamped and reported as an error.  The parity cases (and the
patch-wise continuation path's resummation) run through it (in a subprocess,
as the library is chosen when it is loaded) without an error and give the
plain build's fields."""
import os
import subprocess
import sys
import textwrap

import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb

pytestmark = pytest.mark.gpu

ROOT = os.path.dirname(os.path.dirname(os.path.abspath(__file__)))

CASES = textwrap.dedent('''
    import math, sys
    import numpy as np
    from paper_2301_03814_gb300 import swkb, workloads as w
    out = sys.argv[1]
    M, F = swkb.SWKB_MIXED, swkb.SWKB_FP64
    duct = w.config_surface_duct_small(n_screens=2)
    pr = duct.profile
    two_col = duct.with_(profile=w._table([0.0, 50.0], pr.z0, pr.dz, pr.n_p,
                         [w.f_trilinear_duct(12.0, -0.1), w.f_trilinear_duct(15.0, -0.1)]))
    res = {}
    res["c1_fp64"] = swkb.Plan(w.config_unit_periodic(n_screens=3), F).propagate()
    res["c1_mixed"] = swkb.Plan(w.config_unit_periodic(n_screens=3), M).propagate()
    res["duct_fp64"] = swkb.Plan(duct, F).propagate()
    res["duct_mixed_snap"] = swkb.Plan(duct, M).propagate(snapshot_every=1)
    res["two_column_mixed"] = swkb.Plan(two_col, M).propagate()
    res["planes"] = swkb.Plan(w.config_unit_periodic(n_screens=2), M, planes=4).propagate_planes(4)
    res["n64"] = swkb.Plan(w.config_homogeneous(eps0=1.05, n_z=64, height=32.0, ray_stride=1,
                                                rk4_steps=3), M).propagate()
    res["n2p20"] = swkb.Plan(w.config_homogeneous(eps0=1.02, n_z=1 << 20, height=32.0,
                                                  ray_stride=64, rk4_steps=2, n_screens=2,
                                                  theta_deg=20.0), M).propagate()
    res["one_mode"] = swkb.Plan(duct.with_(theta_max=math.radians(0.02)), M).propagate()
    res["paper_scale"] = swkb.Plan(w.config_range_dependent_duct(n_screens=3, range_m=150.0,
                                                                 col_every_m=50.0),
                                   M).propagate()
    # patch-wise continuation (open interval): ragged tail past the last
    # patch, ray strides 1 and 8, both precisions
    opn = w.config_open_lens(n_z=8192, fc_patch=910, fc_overlap=248, n_screens=2)
    res["open_mixed"] = swkb.Plan(opn, M).propagate()
    res["open_fp64_R1"] = swkb.Plan(w.config_open_lens(n_z=8192, fc_patch=910, fc_overlap=248,
                                                       n_screens=2, ray_stride=1),
                                    F).propagate()
    np.savez(out, **res)
''')


def _run(env_extra, path):
    env = dict(os.environ, **env_extra)
    r = subprocess.run([sys.executable, "-c", CASES, path], cwd=ROOT, env=env,
                       capture_output=True, text=True, timeout=1200)
    assert r.returncode == 0, r.stderr[-3000:]
    return np.load(path)


def test_checked_build_runs_the_parity_cases_in_bounds(tmp_path):
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    from paper_2301_03814_gb300 import build
    build.build(checked=True)
    plain = _run({"SWKB_CHECKED": "0"}, str(tmp_path / "plain.npz"))
    checked = _run({"SWKB_CHECKED": "1"}, str(tmp_path / "checked.npz"))
    for k in plain.files:
        a, b = plain[k], checked[k]
        tol = 1e-12 if "fp64" in k else 1e-6
        assert np.linalg.norm(a - b) <= tol * np.linalg.norm(a), k
