"""Pins of the Fourier-continuation oracle (Sec. 2.2, Eq. ifft_eq_phi_patches).

Each check compares the oracle with something other than itself: the
mathematics of the Gram basis, exact polynomials, a smooth function's own
values between grid points, the defining identities of a partition of unity,
the exact propagator of a homogeneous medium (the angular spectrum, Sec. 2.1,
whose plane waves are exact solutions), and the periodic S-WKB oracle on a
field that never reaches the interval's ends.  Every pin takes the pieces it
checks as arguments, so that the planted-mistake tests can hand it altered
copies."""
import math

import numpy as np

from paper_2301_03814_gb300 import workloads as w

K = 2.0 * math.pi          # unit wavelength
STEP = 1.0 / 3.0           # grid step: three points per wavelength


def series(e: np.ndarray, xx: np.ndarray) -> np.ndarray:
    """The full N_p-periodic Fourier series of the sequence e (every DFT
    bin, frequencies -N_p/2 .. N_p/2 - 1) at grid-unit positions xx."""
    n_p = len(e)
    wv = np.fft.fft(e)
    nn = np.fft.fftfreq(n_p, 1.0 / n_p)
    return (np.exp(2j * np.pi * np.outer(xx, nn) / n_p) @ wv) / n_p


def _offgrid(n):
    xx = np.arange(4 * (n - 1) + 1) / 4.0
    return xx, xx / (n - 1)


def pin_gram_basis(Q):
    """Q's columns are the Gram polynomials on the points 0..d-1: orthonormal,
    column j orthogonal to every monomial of degree < j (so it has degree j),
    column 0 constant."""
    d = Q.shape[0]
    x = np.arange(d, dtype=np.float64)
    assert np.max(np.abs(Q.T @ Q - np.eye(d))) < 1e-13
    for j in range(d):
        for k in range(j):
            mono = x ** k
            assert abs(mono @ Q[:, j]) < 1e-12 * np.linalg.norm(mono)
    assert np.ptp(Q[:, 0]) < 1e-15 and abs(abs(Q[0, 0]) - 1.0 / math.sqrt(d)) < 1e-15


def pin_polynomials_reproduced(extend, Q, A, n=64, tol=1e-9):
    """Every polynomial of degree < d is matched exactly by its Gram
    expansion, so its continuation is the blend of the polynomial itself and
    the series reproduces it between the grid points (to the blend fit)."""
    d = Q.shape[0]
    x = np.arange(n) / (n - 1)
    xx, xe = _offgrid(n)
    for deg in range(d):
        got = series(extend((2.0 * x - 1.0) ** deg, Q, A), xx)
        assert np.max(np.abs(got - (2.0 * xe - 1.0) ** deg)) < tol, deg


def pin_smooth_convergence(extend, Q, A):
    """A smooth non-periodic function: the series between grid points
    converges at high order (FC-Gram with d = 5 is fifth order; at least
    fourth is required) and reaches 1e-8 with 128 points on [0, 1]."""
    def g(x):
        return np.exp(np.sin(3.0 * x)) + x ** 3
    errs = []
    for n in (32, 64, 128):
        x = np.arange(n) / (n - 1)
        xx, xe = _offgrid(n)
        errs.append(np.max(np.abs(series(extend(g(x), Q, A), xx) - g(xe))))
    assert errs[2] < 1e-8, errs
    assert errs[0] / errs[1] > 16.0 and errs[1] / errs[2] > 16.0, errs


def pin_periodic_function(extend, Q, A, n=256, tol=1e-6):
    """A function periodic on the patch (whole periods between its first and
    last point; five periods over 256 points) is, to the continuation, just a
    smooth function: reproduced between grid points to 1e-6 (fifth order:
    about 1e-5 with 128 points)."""
    def f(x):
        return np.exp(2j * np.pi * 2.0 * x) + 0.5 * np.sin(2.0 * np.pi * 5.0 * x)
    x = np.arange(n) / (n - 1)
    xx, xe = _offgrid(n)
    assert np.max(np.abs(series(extend(f(x), Q, A), xx) - f(xe))) < tol


def pin_partition(Patches, smooth_step):
    """F1/F2: the weights form a partition of unity on the interval away from
    its ends (at grid points and between them), each vanishes at both ends of
    its own patch and outside it, lies in [0, 1] and is 1 on the patch's
    interior; the step satisfies r(t) + r(1 - t) = 1."""
    t = np.linspace(-0.5, 1.5, 401)
    assert np.max(np.abs(smooth_step(t) + smooth_step(1.0 - t) - 1.0)) < 1e-15
    assert smooth_step(np.array([0.0]))[0] == 0.0 and smooth_step(np.array([1.0]))[0] == 1.0
    for n_z, n_pat, n_ov in ((272, 80, 16), (64, 64, 8), (1000, 200, 100)):
        pt = Patches(n_z, n_pat, n_ov)
        u = np.linspace(-3.0, n_z + 2.0, 7 * n_z + 1)
        S = np.array([pt.weight(p, u) for p in range(pt.P)])
        inside = (u >= n_ov - 1) & (u <= n_z - n_ov)
        assert np.max(np.abs(S.sum(axis=0)[inside] - 1.0)) < 1e-15
        assert S.min() >= 0.0 and S.max() <= 1.0
        assert np.max(S.sum(axis=0)) <= 1.0 + 1e-15
        for p in range(pt.P):
            s, e = pt.start[p], pt.start[p] + n_pat - 1
            assert pt.weight(p, np.array([float(s), float(e)])).max() == 0.0
            outside = (u < s) | (u > e)
            assert np.all(S[p][outside] == 0.0)
            core = (u >= s + n_ov - 1) & (u <= e - n_ov + 1)
            assert np.all(S[p][core] == 1.0)
        # at most two patches overlap anywhere
        assert np.max((S > 0).sum(axis=0)) <= 2


def open_problem(n_pat, n_ov, P, zc, tilt_deg, dx, medium=None, n_screens=1, theta_deg=60.0,
                 rk4_steps=4, ray_stride=1):
    """A non-periodic interval of P patches at three points per wavelength,
    a Gaussian beam (waist 3 wavelengths) centred at zc, and a medium table
    reaching one interval height beyond both ends."""
    n_z = (P - 1) * (n_pat - n_ov) + n_pat
    H = n_z * STEP
    f = medium if medium is not None else w.f_const(1.0)
    dzp = 0.0625
    prof = w._table([0.0], -H, dzp, int(round(3.0 * H / dzp)) + 1, [f])
    z = STEP * np.arange(n_z)
    u0 = w.gaussian_beam(z, K, zc, 3.0, math.radians(tilt_deg))
    return w.Problem(f"open-{P}x{n_pat}", K, 0.0, H, n_z, w.BC_OPEN, 0.0, dx, n_screens, prof,
                     u0, math.radians(theta_deg), ray_stride, rk4_steps, 0.0,
                     fc_patch=n_pat, fc_overlap=n_ov)


def angular_spectrum(u0, dx, eps0=1.0, pad=8):
    """Exact propagation over dx in the homogeneous medium eps0: the field
    (zero beyond the interval, which it never reaches) on a period pad times
    longer, each plane wave multiplied by exp(i k sqrt(eps0 - kappa^2) dx)."""
    n = len(u0)
    ub = np.zeros(pad * n, dtype=np.complex128)
    ub[:n] = u0
    kap = np.fft.fftfreq(pad * n, d=STEP) * (2.0 * math.pi / K)
    prop = np.exp(1j * K * np.sqrt((eps0 - kap ** 2).astype(np.complex128)) * dx)
    return np.fft.ifft(np.fft.fft(ub) * prop)[:n]


def homogeneous_error(FC, n_pat, n_ov, P, zc, tilt_deg, dx):
    pb = open_problem(n_pat, n_ov, P, zc, tilt_deg, dx)
    got = FC(pb).screen(pb.u0, 0)
    want = angular_spectrum(pb.u0, dx)
    return np.max(np.abs(got - want)) / np.max(np.abs(want))


def pin_homogeneous(FC):
    """Homogeneous medium against the angular spectrum, one screen of 5
    wavelengths.  The method's own errors are the interpolation of S^p
    across the stencils and the geometric transport of S^p (Sec. 2.2 puts
    S^p in the launch amplitude), both set by the overlap width: with 48
    points (16 wavelengths) they are below 2e-6 for a beam inside one patch,
    for a tilted beam crossing an overlap, and for one patch alone, and they
    fall by more than 10x from a 32-point to a 48-point overlap."""
    assert homogeneous_error(FC, 144, 48, 3, (96 + 72) * STEP, 5.0, 5.0) < 2e-6
    assert homogeneous_error(FC, 144, 48, 3, (144 - 24) * STEP, 8.0, 5.0) < 2e-6
    assert homogeneous_error(FC, 192, 48, 1, 96 * STEP, -4.0, 5.0) < 2e-6
    e32 = homogeneous_error(FC, 144, 32, 3, (144 - 16) * STEP, 8.0, 5.0)
    e48 = homogeneous_error(FC, 144, 48, 3, (144 - 24) * STEP, 8.0, 5.0)
    assert e32 / e48 > 10.0, (e32, e48)


def pin_against_periodic(FC, Periodic):
    """A Gaussian lens (the paper's eps = 1 + a exp(-b (z - zc)^2)), two
    screens, beam well inside the interval: the patch-wise method agrees with
    the periodic S-WKB on the same grid (a field that never reaches the ends
    does not see the boundary treatment) to the two discretisations' gap."""
    H = ((3 - 1) * (144 - 48) + 144) * STEP
    pb = open_problem(144, 48, 3, 52.0, 6.0, 5.0, medium=w.f_gaussian(0.01, 0.01, zc=H / 2),
                      n_screens=2, rk4_steps=8)
    got = FC(pb).propagate(pb.u0)
    want = Periodic(pb.with_(bc=w.BC_PERIODIC)).propagate(pb.u0)
    assert np.max(np.abs(got - want)) / np.max(np.abs(want)) < 1e-5


def pin_homogeneous_closed_form(FC):
    """In a homogeneous medium every ray of mode n is straight with slope
    t_n = kappa_n / Pbar_n, Pbar_n = sqrt(1 - kappa_n^2), keeps amplitude 1
    (Z_s = 1) and gains phase k Pbar_n dx, so Sec. 2.2's recipe (launch
    amplitude S^p(z) w_n^p / N) has the closed form
        u(z) = sum_p sum_n c_n^p S^p(z - t_n dx) exp(i k (kappa_n (z - a_p) + Pbar_n dx))
    for ANY coefficients c_n^p: S^p is carried along the ray from where it
    started.  The oracle's screen must equal it for a random field up to the
    4-point interpolation of S^p between ray landings (below 1e-6 of the
    sum of the terms' magnitudes with 48-point overlaps; 2e-6 is required)."""
    rng = np.random.default_rng(23)
    pb = open_problem(144, 48, 3, 50.0, 0.0, 7.0)
    n_z = pb.n_z
    u = rng.standard_normal(n_z) + 1j * rng.standard_normal(n_z)
    o = FC(pb)
    got = o.screen(u, 0)
    c = o.patch_modes(u)
    z = STEP * np.arange(n_z)
    want = np.zeros(n_z, dtype=np.complex128)
    scale = np.zeros(n_z)
    for p in range(o.patches.P):
        a_p = pb.z_a + STEP * o.patches.start[p]
        for i, n in enumerate(o.n):
            kap = o.kappa[i]
            pbar = math.sqrt(1.0 - kap * kap)
            S = o.patches.weight(p, (z - kap / pbar * pb.dx - pb.z_a) / STEP)
            term = c[p, i] * S * np.exp(1j * pb.k * (kap * (z - a_p) + pbar * pb.dx))
            want += term
            scale += np.abs(term)
    assert np.max(np.abs(got - want)) < 2e-6 * np.max(scale)


def pin_planes_homogeneous(FC):
    """Fields between screens (planes x_q + j dx / 4): in eps = 1 each plane
    is the angular spectrum over j dx / 4 (same bound as the screen's pin),
    and the last plane is the screen itself."""
    pb = open_problem(144, 48, 3, (144 - 24) * STEP, 8.0, 5.0)
    o = FC(pb)
    fields = o.screen_planes(pb.u0, 0, 4)
    for j, f in enumerate(fields, start=1):
        want = angular_spectrum(pb.u0, j * pb.dx / 4)
        assert np.max(np.abs(f - want)) / np.max(np.abs(want)) < 2e-6, j
    assert np.array_equal(fields[-1], o.screen(pb.u0, 0))
