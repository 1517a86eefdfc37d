"""Pins of the CPU oracle (no GPU).  See oracle_pins.py for what each fixes."""
import math

import numpy as np
import pytest

import oracle_pins as P
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import (CausticError, Medium, Oracle, RangeError, TurningError,
                                absorber, geometry, hermite5)


def test_hermite5_reproduces_quintics():
    rng = np.random.default_rng(3)
    coef = rng.standard_normal(6)
    p = np.polynomial.Polynomial(coef)
    z0, h, n = -1.3, 0.37, 12
    zn = z0 + h * np.arange(n)
    prof = w.Profile(np.array([0.0]), z0, h, p(zn)[None], p.deriv(1)(zn)[None], p.deriv(2)(zn)[None])
    m = Medium(prof, False, 0.0)
    z = rng.uniform(zn[0], zn[-1], 200)
    e, ez, ezz = m.eval(0.0, True, z)
    assert np.max(np.abs(e - p(z))) < 1e-12 * np.max(np.abs(p(z)))
    assert np.max(np.abs(ez - p.deriv(1)(z))) < 1e-11 * np.max(np.abs(p.deriv(1)(z)))
    assert np.max(np.abs(ezz - p.deriv(2)(z))) < 1e-10 * np.max(np.abs(p.deriv(2)(z)))


def test_hermite5_basis_interpolates_data():
    # t = 0 and t = 1 give back the nodal value / derivatives
    for t, want in ((0.0, (1.0, 2.0, 3.0)), (1.0, (4.0, 5.0, 6.0))):
        v = hermite5(1.0, 2.0, 3.0, 4.0, 5.0, 6.0, t, 0.5)
        assert np.allclose(v, want, atol=1e-13)


def test_mirrored_medium_is_reflection():
    pb = w.config_surface_duct_small()
    m = Medium(pb.profile, True, 0.0)
    z = np.linspace(0.3, 40.0, 77)
    a = m.eval(0.0, True, z)
    b = m.eval(0.0, True, -z)
    assert np.array_equal(a[0], b[0]) and np.array_equal(a[1], -b[1]) and np.array_equal(a[2], b[2])


def test_column_weights_left_right_limits():
    pb = w.config_unit_periodic()
    m = Medium(pb.profile, False, 0.0)
    assert m.column_weights(100.0, True) == (2, 0.0)     # right limit: linear half
    assert m.column_weights(100.0, False) == (0, 1.0)    # left limit: homogeneous half
    c, th = m.column_weights(150.0, True)
    assert c == 2 and abs(th - 0.5) < 1e-15
    assert m.column_weights(-5.0, True) == (0, 0.0)
    assert m.column_weights(500.0, False) == (2, 1.0)


def test_x_only_medium_column_blend_and_limits():
    """Linear-in-x blend between range columns and the left / right limits
    at a jump on a screen edge, against closed-form rays (R10)."""
    assert P.pin_x_only_columns(Oracle) < 1e-9


def test_geometry_counts():
    g = geometry(w.config_unit_periodic())
    assert (g.N, g.n_max, g.M, g.G, g.NRT) == (512, 32, 65, 96, 704)
    g = geometry(w.config_surface_duct())
    assert (g.N, g.n_max, g.M, g.R, g.N_r, g.G, g.NRT) == (32768, 488, 977, 16, 2048, 19, 2086)


def test_absorber_values():
    pb = w.config_surface_duct_small()
    g = geometry(pb)
    W = absorber(pb, g)
    H = pb.z_b - pb.z_a
    z = g.z_lo + g.dz * np.arange(g.N)
    assert np.all(W[np.abs(z) <= 0.8 * H] == 1.0)
    i = int(np.argmin(np.abs(np.abs(z) - 0.9 * H)))
    assert abs(W[i] - math.cos(math.pi / 4) ** 2) < 1e-2
    assert W[0] < 1e-12 and np.allclose(W, W[(g.N - np.arange(g.N)) % g.N])


def test_modes_bruteforce():
    assert P.pin_modes_bruteforce(Oracle) < 1e-13


@pytest.mark.parametrize("bc,eps0,R,nt", [(w.BC_PERIODIC, 1.0, 1, 4), (w.BC_PERIODIC, 1.2, 4, 2),
                                         (w.BC_NEUMANN, 1.0, 2, 4), (w.BC_DIRICHLET, 1.05, 1, 3)])
def test_homogeneous_equals_angular_spectrum(bc, eps0, R, nt):
    assert P.pin_homogeneous(Oracle, bc=bc, eps0=eps0, R=R, nt=nt) < 1e-12


def test_linear_ray_closed_form_rk4_order():
    e8 = P.pin_linear_ray(Oracle, 8)
    e16 = P.pin_linear_ray(Oracle, 16)
    e64 = P.pin_linear_ray(Oracle, 64)
    assert e64 < 1e-9
    assert 8.0 < e8 / e16 < 24.0        # fourth order


@pytest.mark.parametrize("xdep", [False, True])
def test_ray_tube_flux_and_jacobian(xdep):
    assert P.pin_tube_flux(Oracle, x_dependent=xdep) < 1e-6


def test_interpolation_stencil_remainder():
    assert P.pin_interp_stencil(Oracle) < 1e-9


@pytest.mark.slow
def test_airy_exact_linear_medium():
    assert P.pin_airy(Oracle) < 1e-4


def test_caustic_is_an_error():
    pb = w.config_gaussian_medium(a=0.05, b=0.01, dx=100.0, n_screens=1)
    with pytest.raises(CausticError):
        Oracle(pb).propagate(pb.u0)


def test_turning_point_is_an_error():
    k = 2 * math.pi
    prof = w._table([0.0, 20.0], -200.0, 0.125, 3201, [w.f_const(1.0), w.f_const(0.5)])
    z = 64.0 / 256 * np.arange(256)
    pb = w.Problem("turn", k, 0.0, 64.0, 256, w.BC_PERIODIC, 0.0, 20.0, 1, prof,
                   w.gaussian_beam(z, k, 32, 3, 0.0), math.radians(60.0), 1, 8)
    with pytest.raises(TurningError):
        Oracle(pb).propagate(pb.u0)


def test_table_range_is_an_error():
    k = 2 * math.pi
    prof = w._table([0.0], -2.0, 0.125, 540, [w.f_const(1.0)])
    z = 64.0 / 256 * np.arange(256)
    pb = w.Problem("short", k, 0.0, 64.0, 256, w.BC_PERIODIC, 0.0, 20.0, 1, prof,
                   w.gaussian_beam(z, k, 32, 3, 0.0), math.radians(30.0), 1, 8)
    with pytest.raises(RangeError):
        Oracle(pb).propagate(pb.u0)


def test_sampled_screen_equals_full_screen():
    """screen_points (rays marched in a window per point) reproduces the full
    screen at sampled points, including points near the domain edges."""
    pb = w.config_surface_duct_small(n_screens=1)
    o = Oracle(pb)
    u = o.extend(pb.u0)
    full = o.screen(u, 2)
    ms = [o.g.N // 2, o.g.N // 2 + 7, o.g.N - 40, 3 * o.g.N // 4 + 123, 100]
    got = o.screen_points(u, 2, ms)
    assert np.max(np.abs(got - full[ms])) < 1e-12 * np.max(np.abs(full))


@pytest.mark.parametrize("bc", [w.BC_PERIODIC, w.BC_NEUMANN, w.BC_DIRICHLET])
def test_planes_between_screens_homogeneous(bc):
    assert P.pin_planes_homogeneous(Oracle, bc) < 1e-12


def test_linear_ray_stopped_inside_the_screen():
    assert P.pin_linear_ray_steps(Oracle) < 1e-7


def test_last_plane_is_the_screen():
    pb = w.config_surface_duct_small(n_screens=2, n_z=1024, height=20.0)
    o = Oracle(pb)
    rows = o.propagate_planes(pb.u0, 0, 2, 4)
    _, snaps = o.propagate(pb.u0, 0, 2, snapshots=True)
    assert np.array_equal(rows[3], snaps[0]) and np.array_equal(rows[7], snaps[1])
    with pytest.raises(ValueError):
        o.screen_planes(o.extend(pb.u0), 0, 3)


def test_planes_inside_a_screen_carry_no_absorber():
    assert P.pin_planes_before_absorber(Oracle) < 1e-12


# -- separation of variables (Sec. 3.1): the exact one-way field of an
#    x-invariant medium, from the Hill-matrix eigen-expansion ------------------

def _gaussian_lens(lam, n_z):
    pb = w.config_gaussian_medium(n_screens=3, dx=10.0, theta_deg=30.0, ray_stride=1,
                                  rk4_steps=16, n_z=n_z)
    k = 2.0 * math.pi / lam
    return pb.with_(k=k, u0=w.gaussian_beam(pb.z_phys, k, 32.0, 4.0, math.radians(2.0)))


def test_hill_reference_is_the_angular_spectrum_in_a_homogeneous_medium():
    from refs import angular_spectrum, hill_one_way
    pb = w.config_homogeneous(eps0=1.05, n_z=256, height=32.0)
    g = geometry(pb)
    ref = hill_one_way(pb.u0, pb.k, g.L, lambda t: np.full_like(t, 1.05), 45.0, 127)
    assert P.rel_l2(ref, angular_spectrum(pb.u0, pb.k, g.L, 45.0, 127, 1.05)) < 1e-12


def test_method_error_against_separation_of_variables_shrinks_with_k():
    """S-WKB is asymptotic in k: against the exact field its error is small
    and falls as the wavelength shrinks (measured 3.6e-5 at lambda = 1,
    1.5e-5 at 0.5, 7.1e-6 at 0.25 after 30 m of a Gaussian lens)."""
    from refs import hill_one_way
    f = w.f_gaussian(0.02, 0.01, zc=32.0)
    errs = []
    for lam, n_z in ((1.0, 256), (0.5, 512)):
        pb = _gaussian_lens(lam, n_z)
        g = geometry(pb)
        got = Oracle(pb).propagate(pb.u0)
        ref = hill_one_way(pb.u0, pb.k, g.L, lambda t: f(t)[0], pb.dx * pb.n_screens,
                           int(1.3 * g.L / lam))
        errs.append(P.rel_l2(got, ref))
    assert errs[0] < 1e-4 and errs[1] < 0.7 * errs[0], errs


def test_method_error_against_separation_of_variables_grounded_duct():
    """Neumann ground (mirrored period, even eps), 200 m of the surface duct
    without the absorber: S-WKB within 1e-4 of the exact field (2.1e-5)."""
    from refs import hill_one_way
    pb = w.config_surface_duct_small(n_screens=4).with_(absorber_frac=0.0)
    g = geometry(pb)
    f = w.f_trilinear_duct(pb.meta["z_t"], pb.meta["g_d"])
    n = pb.n_z
    full = np.zeros(2 * n, complex)
    full[n:] = pb.u0
    full[n - np.arange(1, n)] = pb.u0[1:]
    ref = hill_one_way(full, pb.k, g.L, lambda t: f(np.abs(g.z_lo + t - pb.z_a))[0],
                       pb.dx * pb.n_screens, 300, n_quad=16384)[n:]
    assert P.rel_l2(Oracle(pb).propagate(pb.u0), ref) < 1e-4
