"""The GPU path against the exact one-way field of x-invariant media from
separation of variables (Sec. 3.1; refs.hill_one_way, pinned to the angular
spectrum).  This measures the method's own error, not parity with the
oracle: S-WKB is asymptotic in k, so the bounds are the method's, with the
measured values in the docstrings."""
import math

import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import geometry, rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _mirrored(u):
    n = len(u)
    full = np.zeros(2 * n, complex)
    full[n:] = u
    full[n - np.arange(1, n)] = u[1:]
    return full


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_gaussian_lens_against_separation_of_variables(prec):
    """k = 2 pi, 30 m of eps = 1 + 0.02 exp(-0.01 (z - 32)^2): measured
    3.6e-5 at both precisions (the oracle's own error)."""
    from refs import hill_one_way
    pb = w.config_gaussian_medium(n_screens=3, dx=10.0, theta_deg=30.0, ray_stride=1,
                                  rk4_steps=16)
    pb = pb.with_(u0=w.gaussian_beam(pb.z_phys, pb.k, 32.0, 4.0, math.radians(2.0)))
    g = geometry(pb)
    f = w.f_gaussian(0.02, 0.01, zc=32.0)
    ref = hill_one_way(pb.u0, pb.k, g.L, lambda t: f(t)[0], 30.0, 83)
    err = rel_l2(swkb.Plan(pb, prec).propagate(), ref)
    print(f"gaussian lens, precision {prec}: {err:.3e}")
    assert err < 1e-4


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_full_size_duct_against_separation_of_variables(prec):
    """The 16384-point surface duct (lambda = 5 cm, 200 m, Neumann ground),
    without its absorber, over the first 2 km (40 screens; the beam stays
    far below the top): measured 5.0e-5 against the exact field of the
    mirrored period at both precisions."""
    from refs import hill_one_way
    pb = w.config_surface_duct(n_screens=40, range_m=2000.0).with_(absorber_frac=0.0)
    g = geometry(pb)
    f = w.f_trilinear_duct(pb.meta["z_t"], pb.meta["g_d"])
    n = pb.n_z
    ref = hill_one_way(_mirrored(pb.u0), pb.k, g.L,
                       lambda t: f(np.abs(g.z_lo + t - pb.z_a))[0],
                       pb.dx * pb.n_screens, 640, n_quad=1 << 16)[n:]
    err = rel_l2(swkb.Plan(pb, prec).propagate(), ref)
    print(f"16384-point duct, 2 km, precision {prec}: {err:.3e}")
    assert err < 2e-4


def _layer_reference(pb, x, extra=100):
    from refs import hill_one_way
    g = geometry(pb)
    a, b = pb.meta["a"], pb.meta["b"]
    return hill_one_way(pb.u0, pb.k, g.L, lambda t: 1.0 + a * np.exp(-b * (t - g.L / 2) ** 2),
                        x, g.n_max + extra, n_quad=8192)


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_gaussian_lens_40km_against_separation_of_variables(prec):
    """Like the paper's first example (a single focus): eps = 1 + 1e-4
    exp(-1e-4 z^2), lambda = 5 cm, 401 modes, 40 km in 40 screens of 1 km.
    Measured 5.4e-5 (FP64) and 5.6e-5 (mixed); mixed 1.7 ms."""
    import time
    pb = w.config_gaussian_lens_40km()
    ref = _layer_reference(pb, pb.dx * pb.n_screens)
    plan = swkb.Plan(pb, prec)
    plan.propagate(n_screens=1)
    t = time.perf_counter()
    got = plan.propagate()
    dt = time.perf_counter() - t
    err = rel_l2(got, ref)
    print(f"40 km lens, precision {prec}: rel-L2 {err:.3e}, {dt * 1e3:.1f} ms "
          f"({pb.n_z * pb.n_screens / dt:.3e} screen-points/s)")
    assert err < 2e-4


def test_gaussian_duct_200km_error_falls_with_screen_spacing():
    """Like the paper's second example (a narrow duct, the beam bouncing ten
    times): 200 km with screens every 1000, 500 and 250 m, mixed path; the
    error against the exact field falls with the spacing (measured 2.6e-2,
    5.7e-3, 7.5e-4: about the cube of the spacing; 29 ms for 800 screens)."""
    import time
    base = w.config_gaussian_duct_200km()
    ref = _layer_reference(base, 200_000.0)
    errs = []
    for n in (200, 400, 800):
        pb = base.with_(n_screens=n, dx=200_000.0 / n)
        plan = swkb.Plan(pb, swkb.SWKB_MIXED)
        plan.propagate(n_screens=1)
        t = time.perf_counter()
        got = plan.propagate()
        dt = time.perf_counter() - t
        errs.append(rel_l2(got, ref))
        print(f"200 km duct, {n} screens of {pb.dx:.0f} m: rel-L2 {errs[-1]:.3e}, "
              f"{dt * 1e3:.1f} ms")
    assert errs[0] > 2.0 * errs[1] > 4.0 * errs[2] and errs[2] < 2e-3


def test_error_curve_against_the_gpu_reference():
    """The same 200 km curve with the reference computed on the GPU
    (swkb_hill_propagate, the separation-of-variables solver of Sec. 3.1):
    it equals the CPU reference to the phase conditioning of a 200 km range
    (1e-6), so the S-WKB errors agree with those above, and the whole
    experiment runs on the GPU."""
    base = w.config_gaussian_duct_200km()
    cpu_ref = _layer_reference(base, 200_000.0)
    hi = w.hill_gaussian_duct_200km()
    d = swkb.hill_desc(hi.bc, hi.z_a, hi.z_b, hi.n_z, hi.K, hi.n_q, z_sym=hi.z_c)
    gpu_ref = swkb.swkb_hill_propagate(d, hi.k, hi.eps, hi.u0, hi.xs)[0, 0]
    assert rel_l2(gpu_ref, cpu_ref) < 1e-6
    for n in (200, 800):
        got = swkb.Plan(base.with_(n_screens=n, dx=200_000.0 / n), swkb.SWKB_MIXED).propagate()
        e_gpu, e_cpu = rel_l2(got, gpu_ref), rel_l2(got, cpu_ref)
        assert abs(e_gpu - e_cpu) < 1e-3 * e_cpu + 1e-6, (n, e_gpu, e_cpu)


def test_lens_40km_against_the_gpu_reference():
    """The 40 km lens (E1-like) against the GPU reference: the same
    5.4e-5 / 5.6e-5 error as against the CPU reference."""
    pb = w.config_gaussian_lens_40km()
    cpu_ref = _layer_reference(pb, pb.dx * pb.n_screens)
    hi = w.hill_gaussian_lens_40km()
    d = swkb.hill_desc(hi.bc, hi.z_a, hi.z_b, hi.n_z, hi.K, hi.n_q, z_sym=hi.z_c)
    gpu_ref = swkb.swkb_hill_propagate(d, hi.k, hi.eps, hi.u0, hi.xs)[0, 0]
    assert rel_l2(gpu_ref, cpu_ref) < 1e-7
    got = swkb.Plan(pb, swkb.SWKB_MIXED).propagate()
    assert rel_l2(got, gpu_ref) < 2e-4
