"""Pins of the CPU oracle against facts fixed outside it.

Each function runs one check against a given oracle class and returns the
measured error, so that the same checks serve the plain pin tests and the
mutation tests (which plant a mistake in a subclass and expect a pin to
fail).  None of these re-types the oracle's formulas: the references are
closed forms, brute-force sums, exact Helmholtz solutions or conservation laws.
"""
from __future__ import annotations

import math

import numpy as np

from paper_2301_03814_gb300 import workloads as w
from refs import airy_field, angular_spectrum, linear_ray
from oracle.swkb_oracle import rel_l2


def _linear_problem(a, dx, nt, eps0=1.0):
    k = 2.0 * math.pi
    prof = w._table([0.0], -64.0, 0.125, int(256 / 0.125) + 1, [w.f_linear(eps0, a)])
    z = 64.0 / 512 * np.arange(512)
    return w.Problem("linear", k, 0.0, 64.0, 512, w.BC_PERIODIC, 0.0, dx, 1, prof,
                     np.zeros(512, complex), math.radians(30.0), 1, nt, 0.0)


def pin_modes_bruteforce(O, N=24, seed=0):
    """DFT by a direct double loop over m and n (definition of Eq. fft_eq
    with the reading R1), and a single plane wave mapping to one mode."""
    rng = np.random.default_rng(seed)
    pb = w.config_homogeneous(n_z=N, height=N * 0.125, dx=1.0, n_screens=1, theta_deg=60)
    o = O(pb)
    u = rng.standard_normal(N) + 1j * rng.standard_normal(N)
    c = o.modes(u)
    err = 0.0
    for i, n in enumerate(o.n):
        s = 0j
        for m in range(N):
            s += u[m] * complex(math.cos(2 * math.pi * n * m / N), -math.sin(2 * math.pi * n * m / N))
        err = max(err, abs(c[i] - s / N))
    n0 = int(o.n[-2])
    pw = np.exp(2j * math.pi * n0 * np.arange(N) / N)
    c = o.modes(pw)
    want = (o.n == n0).astype(float)
    return max(err, float(np.max(np.abs(c - want))))


def pin_homogeneous(O, bc=w.BC_PERIODIC, eps0=1.0, R=1, n_z=256, nt=4):
    """Homogeneous medium: S-WKB must equal the band-limited angular-spectrum
    propagator (rays straight, A constant, residual phase constant)."""
    pb = w.config_homogeneous(eps0=eps0, n_z=n_z, dx=15.0, n_screens=3, bc=bc,
                              ray_stride=R, rk4_steps=nt)
    o = O(pb)
    got = o.propagate(pb.u0)
    g = o.g
    if bc == w.BC_PERIODIC:
        ref = angular_spectrum(pb.u0, pb.k, g.L, pb.dx * pb.n_screens, g.n_max, eps0)
    else:
        sgn = 1.0 if bc == w.BC_NEUMANN else -1.0
        full = np.zeros(2 * n_z, complex)
        full[n_z:] = pb.u0
        full[n_z - np.arange(1, n_z)] = sgn * pb.u0[1:]
        ref = angular_spectrum(full, pb.k, g.L, pb.dx * pb.n_screens, g.n_max, eps0)[n_z:]
    return rel_l2(got, ref)


def pin_linear_ray(O, nt):
    """Rays of eps = 1 + a z against their closed form; returns the largest
    relative error of (z - s, Q, r, Z_s, Q_s) over a set of launches."""
    a, dx = 0.01, 20.0
    pb = _linear_problem(a, dx, nt)
    o = O(pb)
    kap = np.array([-0.3, -0.1, 0.0, 0.15, 0.4])
    s = np.array([-5.0, 3.0, 10.0, 20.0, 33.0])
    got = o.march(0, kap, s)
    err = 0.0
    for i in range(len(kap)):
        ref = linear_ray(kap[i], s[i], a, dx)
        for key, scale in (("z", abs(ref["z"] - s[i]) + 1.0), ("Q", 1.0), ("r", abs(ref["r"])),
                           ("Zs", 1.0), ("Qs", abs(ref["Qs"]) + 1e-12)):
            g = got[key][i] - (0.0 if key != "z" else 0.0)
            err = max(err, abs(g - ref[key]) / scale)
        # amplitude: P conserved in an x-invariant medium, so a = 1/sqrt(Z_s)
        err = max(err, abs(got["a"][i] - 1.0 / math.sqrt(ref["Zs"])))
    return err


def pin_tube_flux(O, ds=0.01, x_dependent=False):
    """Gaussian lens eps = 1 + a exp(-b (z - 32)^2) (paper's exponential
    model).  (i) Z_s and Q_s equal central differences of the landing z and Q
    over the launch coordinate s; (ii) the transport equation in divergence
    form div(A^2 grad psi) = 0, integrated over a ray tube, conserves the
    x-flux A^2 P times the tube width: A1^2 P1 (z1[j+1]-z1[j-1]) =
    A0^2 P0 (s[j+1]-s[j-1]) with A0 = 1.  Returns the largest relative error."""
    pb = w.config_gaussian_medium(a=0.05, b=0.01, dx=20.0, rk4_steps=64)
    if x_dependent:
        # eps varies along x as well (two columns), so P changes on the ray
        pr = pb.profile
        pb = pb.with_(profile=w._table([0.0, 20.0], pr.z0, pr.dz, pr.n_p,
                                       [w.f_gaussian(0.05, 0.01, zc=32.0),
                                        w.f_gaussian(0.09, 0.014, zc=30.0)]))
    o = O(pb)
    s = np.arange(20.0, 44.0, ds)
    err = 0.0
    for kap in (-0.1, 0.0, 0.12):
        r = o.march(0, np.full_like(s, kap), s)
        fd_zs = (r["z"][2:] - r["z"][:-2]) / (2 * ds)
        fd_qs = (r["Q"][2:] - r["Q"][:-2]) / (2 * ds)
        err = max(err, float(np.max(np.abs(fd_zs - r["Zs"][1:-1]))))
        err = max(err, float(np.max(np.abs(fd_qs - r["Qs"][1:-1]))) * 10.0)
        flux1 = r["a"][1:-1] ** 2 * r["P1"][1:-1] * (r["z"][2:] - r["z"][:-2])
        flux0 = r["P0"][1:-1] * 2 * ds
        err = max(err, float(np.max(np.abs(flux1 / flux0 - 1.0))))
    return err


def pin_interp_stencil(O, seed=1):
    """Lagrange remainder of exp on the bracket stencil j-1..j+2:
    24 (f - p) / prod(m - x_i) must lie between min and max of exp over the
    stencil.  This fixes the stencil and the bracket rule, not only the
    polynomial degree."""
    rng = np.random.default_rng(seed)
    pb = w.config_homogeneous(n_z=64, height=8.0, dx=1.0, n_screens=1, theta_deg=30)
    o = O(pb)
    N = o.g.N
    nodes = np.cumsum(rng.uniform(0.6, 1.4, N + 40)) - 20.0
    scale = 0.25
    f = np.exp(scale * nodes)
    (p,) = o.interpolate(nodes, (f,))
    m = np.arange(N, dtype=float)
    j = np.searchsorted(nodes, m, side="right") - 1
    xs = [nodes[j + q] for q in (-1, 0, 1, 2)]
    prod = np.prod([m - x for x in xs], axis=0)
    ok = np.abs(prod) > 1e-9
    ratio = 24.0 * (np.exp(scale * m) - p)[ok] / prod[ok] / scale ** 4
    lo = np.exp(scale * xs[0][ok])
    hi = np.exp(scale * xs[3][ok])
    viol = np.maximum(lo * (1 - 1e-6) - ratio, 0) + np.maximum(ratio - hi * (1 + 1e-6), 0)
    return float(np.max(viol / hi))


def pin_airy(O):
    """Full S-WKB in eps = 1 + 1e-3 z against the exact one-way Helmholtz
    field (Airy-function modes), 5 screens of 20 lambda, k = 2 pi."""
    k, a = 2.0 * math.pi, 1e-3
    z = 64.0 / 512 * np.arange(512)
    u0 = w.gaussian_beam(z, k, 32.0, 8.0, math.radians(2.0))
    prof = w._table([0.0], -48.0, 0.125, int(160 / 0.125) + 1, [w.f_linear(1.0, a)])
    pb = w.Problem("airy", k, 0.0, 64.0, 512, w.BC_PERIODIC, 0.0, 20.0, 5, prof, u0,
                   math.radians(30.0), 1, 8, 0.0)
    got = O(pb).propagate(u0)
    ref = airy_field(u0, z, k, a, 100.0, np.arange(-130.0, 105.0, 0.04))
    return rel_l2(got, ref)


def pin_planes_homogeneous(O, bc=w.BC_PERIODIC, planes=4, eps0=1.03):
    """Fields between screens in a homogeneous medium: plane j of screen q
    must equal the band-limited angular spectrum over (q + j / planes) dx."""
    pb = w.config_homogeneous(eps0=eps0, n_z=128, height=32.0, dx=15.0, n_screens=2, bc=bc,
                              ray_stride=1, rk4_steps=8)
    o = O(pb)
    rows = o.propagate_planes(pb.u0, 0, pb.n_screens, planes)
    g = o.g
    err = 0.0
    for q in range(pb.n_screens):
        for j in range(1, planes + 1):
            d = (q + j / planes) * pb.dx
            if bc == w.BC_PERIODIC:
                ref = angular_spectrum(pb.u0, pb.k, g.L, d, g.n_max, eps0)
            else:
                sgn = 1.0 if bc == w.BC_NEUMANN else -1.0
                n = pb.n_z
                full = np.zeros(2 * n, complex)
                full[n:] = pb.u0
                full[n - np.arange(1, n)] = sgn * pb.u0[1:]
                ref = angular_spectrum(full, pb.k, g.L, d, g.n_max, eps0)[n:]
            err = max(err, rel_l2(rows[q * planes + j - 1], ref))
    return err


def pin_linear_ray_steps(O, nt=8):
    """Rays of eps = 1 + a z stopped after k of nt RK4 steps against their
    closed form at x = k dx / nt (the state and amplitude on a plane inside
    the screen)."""
    a, dx = 0.01, 20.0
    pb = _linear_problem(a, dx, nt)
    o = O(pb)
    kap = np.array([-0.3, 0.0, 0.4])
    s = np.array([-5.0, 10.0, 33.0])
    err = 0.0
    for k in (1, nt // 2, nt - 1):
        got = o.march(0, kap, s, steps=k)
        for i in range(len(kap)):
            ref = linear_ray(kap[i], s[i], a, dx * k / nt)
            for key, scale in (("z", abs(ref["z"] - s[i]) + 1.0), ("Q", 1.0),
                               ("r", abs(ref["r"])), ("Zs", 1.0)):
                err = max(err, abs(got[key][i] - ref[key]) / scale)
            err = max(err, abs(got["a"][i] - 1.0 / math.sqrt(ref["Zs"])))
    return err


def pin_planes_before_absorber(O, planes=4):
    """With a top absorber, the planes inside the first screen still carry
    the unabsorbed field: plane j equals the angular spectrum of u0 over
    j dx / planes (the absorber acts only on screens)."""
    pb = w.config_homogeneous(eps0=1.0, n_z=128, height=32.0, dx=15.0, n_screens=1,
                              ray_stride=1, rk4_steps=8).with_(absorber_frac=0.3)
    o = O(pb)
    rows = o.propagate_planes(pb.u0, 0, 1, planes)
    g = o.g
    err = 0.0
    for j in range(1, planes):
        ref = angular_spectrum(pb.u0, pb.k, g.L, j * pb.dx / planes, g.n_max, 1.0)
        err = max(err, rel_l2(rows[j - 1], ref))
    return err


def x_only_ray(kappa, s, eps_a, slope, x):
    """Closed-form ray of a permittivity that depends on x only, linear on the
    stretch ridden, eps = eps_a + slope x (x from the launch): eps_z = 0 keeps
    Q = kappa and Q_s = 0, so Z_s = 1; with P(x) = sqrt(eps(x) - kappa^2),
    z - s = int kappa / P dx, r = int (eps - kappa Q) / P dx = int P dx and the
    amplitude factor is sqrt(P0 / P1)."""
    P0 = math.sqrt(eps_a - kappa * kappa)
    P1 = math.sqrt(eps_a + slope * x - kappa * kappa)
    if slope == 0.0:
        dz, r = kappa * x / P0, P0 * x
    else:
        dz = 2.0 * kappa * (P1 - P0) / slope
        r = 2.0 * (P1 ** 3 - P0 ** 3) / (3.0 * slope)
    return dict(z=s + dz, Q=kappa, r=r, Zs=1.0, Qs=0.0, a=math.sqrt(P0 / P1))


# eps of the two-screen x-only medium: columns at x = 0, D, D, 2 D (a jump at
# the screen edge D: left limit first, then the right limit)
X_ONLY_D = 20.0
X_ONLY_EPS = (1.0, 1.06, 0.97, 1.012)


def pin_x_only_columns(O, nt=64):
    """Range-column weights and limits (reading R10) against closed forms.
    The medium varies with x only, linearly between four columns at
    x = 0, D, D, 2 D with a jump at D; screen 0 rides 0 -> D, screen 1
    D -> 2 D.  Rays are stopped on the planes D/4, D/2, 3D/4 of each screen,
    where eps comes from interior blends of two columns (a swapped blend
    weight makes the profile run backwards there), and at the screen end, where
    screen 0 must take the left limit of the jump and screen 1 start from the
    right limit.  Returns the largest relative error of z - s, Q, r, Z_s, Q_s
    and the amplitude factor."""
    D = X_ONLY_D
    k = 2.0 * math.pi
    cols = [w.f_const(e) for e in X_ONLY_EPS]
    prof = w._table([0.0, D, D, 2 * D], -64.0, 0.125, int(256 / 0.125) + 1, cols)
    pb = w.Problem("x-only", k, 0.0, 64.0, 512, w.BC_PERIODIC, 0.0, D, 2, prof,
                   np.zeros(512, complex), math.radians(30.0), 1, nt, 0.0)
    o = O(pb)
    kap = np.array([-0.4, -0.1, 0.0, 0.2, 0.45])
    s = np.array([-5.0, 3.0, 10.0, 20.0, 33.0])
    err = 0.0
    for q, (ea, eb) in enumerate(((X_ONLY_EPS[0], X_ONLY_EPS[1]),
                                  (X_ONLY_EPS[2], X_ONLY_EPS[3]))):
        slope = (eb - ea) / D
        for steps in (nt // 4, nt // 2, 3 * nt // 4, nt):
            got = o.march(q, kap, s, steps=steps)
            x = D * steps / nt
            for i in range(len(kap)):
                ref = x_only_ray(kap[i], s[i], ea, slope, x)
                for key, scale in (("z", abs(ref["z"] - s[i]) + 1.0), ("Q", 1.0),
                                   ("r", abs(ref["r"])), ("Zs", 1.0), ("Qs", 1.0),
                                   ("a", 1.0)):
                    err = max(err, abs(got[key][i] - ref[key]) / scale)
    return err
