"""Seeded synthetic workloads for the screened-WKB propagator.

This module only *builds inputs*: permittivity tables eps(x, z) with their
first two z-derivatives sampled at uniform nodes, incident fields on the first
screen, and the run parameters of each workload.  It contains none of the
propagation arithmetic (no FFT, no ray march, no interpolation, no resum), so
that the CUDA library and the CPU oracle can both be fed from it without
sharing any of the method's code.

Physical models used (all synthetic, all seeded):

* homogeneous / linear / Gaussian permittivity -- the Gaussian model is the
  paper's exponential permittivity (Sec. 3, Eq. gaussian_permittivity) and the
  super-refractive one its Eq. atmospheric_permittivity;
* a trilinear modified-refractivity profile M(z) for surface ducts, converted
  with eps = (1 + 1e-6 M)^2 (standard earth-flattened modified index; the paper
  does not give one).  Its kinks are rounded over +-1 m with a C^2 blend so that
  eps_zz exists, and for ground-reflected domains it is continued below 1 m by
  an even quartic so that the mirrored profile eps(|z|) is C^2 at z = 0;
* a tilted Gaussian beam (Sec. 3, Eq. inc_field, with a stated waist) and a
  Gaussian antenna pattern of given half-power beamwidth.

Tables are row-major [n_cols][n_p] float64.  Column c sits at range x_cols[c];
two columns at the same x encode a jump (left limit first, then right limit).
"""
from __future__ import annotations

import math
from dataclasses import dataclass, field, replace

import numpy as np

BC_PERIODIC = 0
BC_NEUMANN = 1
BC_DIRICHLET = 2
BC_OPEN = 3        # non-periodic, field vanishing near both ends (patch-wise continuation)


@dataclass
class Profile:
    """eps(x, z) samples: columns at x_cols, nodes z0 + i*dz, i < n_p."""
    x_cols: np.ndarray
    z0: float
    dz: float
    eps: np.ndarray
    eps_z: np.ndarray
    eps_zz: np.ndarray

    @property
    def n_cols(self) -> int:
        return int(self.eps.shape[0])

    @property
    def n_p(self) -> int:
        return int(self.eps.shape[1])

    def nodes(self) -> np.ndarray:
        return self.z0 + self.dz * np.arange(self.n_p)


@dataclass
class Problem:
    """One propagation job: medium, domain, incident field and run parameters.

    z_a, z_b   physical vertical extent; n_z points z_a + m*(z_b-z_a)/n_z.
    bc         BC_PERIODIC: period [z_a, z_b); BC_NEUMANN/BC_DIRICHLET: ground
               at z_a, solved on the mirrored period [2 z_a - z_b, z_b);
               BC_OPEN: [z_a, z_b) is not periodic and the field vanishes near
               both ends; it is expanded patch by patch (fc_patch points per
               patch, fc_overlap shared by neighbours).
    x0, dx     first screen position and screen spacing.
    theta_max  largest kept plane-wave angle (radians); n_max overrides if > 0.
    """
    name: str
    k: float
    z_a: float
    z_b: float
    n_z: int
    bc: int
    x0: float
    dx: float
    n_screens: int
    profile: Profile
    u0: np.ndarray
    theta_max: float
    ray_stride: int
    rk4_steps: int
    absorber_frac: float = 0.0
    n_max: int = 0
    fc_patch: int = 0      # BC_OPEN: grid points per continuation patch
    fc_overlap: int = 0    # BC_OPEN: grid points shared by neighbouring patches
    meta: dict = field(default_factory=dict)

    def with_(self, **kw) -> "Problem":
        return replace(self, **kw)

    @property
    def z_phys(self) -> np.ndarray:
        return self.z_a + (self.z_b - self.z_a) / self.n_z * np.arange(self.n_z)


# ----------------------------------------------------------------------------
# permittivity tables
# ----------------------------------------------------------------------------

def _table(x_cols, z0, dz, n_p, cols):
    """cols: list of callables z -> (eps, eps_z, eps_zz)."""
    z = z0 + dz * np.arange(n_p)
    e = np.empty((len(cols), n_p))
    ez = np.empty_like(e)
    ezz = np.empty_like(e)
    for c, f in enumerate(cols):
        e[c], ez[c], ezz[c] = f(z)
    return Profile(np.asarray(x_cols, dtype=np.float64), float(z0), float(dz), e, ez, ezz)


def f_const(eps0):
    return lambda z: (np.full_like(z, eps0), np.zeros_like(z), np.zeros_like(z))


def f_linear(eps0, a):
    """eps = eps0 + a z."""
    return lambda z: (eps0 + a * z, np.full_like(z, a), np.zeros_like(z))


def f_gaussian(a, b, base=1.0, sign=1.0, zc=0.0):
    """eps = base + sign * a * exp(-b (z - zc)^2)  (paper's Gaussian models)."""
    def f(z):
        y = z - zc
        g = sign * a * np.exp(-b * y * y)
        return base + g, -2.0 * b * y * g, (4.0 * b * b * y * y - 2.0 * b) * g
    return f


def _s(t):
    t = np.clip(t, 0.0, 1.0)
    return t * t * (3.0 - 2.0 * t)


def _s_int(t):
    tc = np.clip(t, 0.0, 1.0)
    return tc ** 3 - 0.5 * tc ** 4 + np.maximum(t - 1.0, 0.0)


def _s_d(t):
    inside = (t > 0.0) & (t < 1.0)
    return np.where(inside, 6.0 * t * (1.0 - t), 0.0)


def modified_refractivity(z, M0, g0, kinks, w=1.0):
    """Piecewise-linear M(z) with slope g0 at z=0 and slope changes
    kinks = [(z_k, dg_k)], each rounded over [z_k - w, z_k + w] by a cubic
    smoothstep in M' (so M is C^2).  Returns M, M', M''."""
    M = M0 + g0 * z
    Mp = np.full_like(z, g0)
    Mpp = np.zeros_like(z)
    for zk, dg in kinks:
        t = (z - zk + w) / (2.0 * w)
        M = M + dg * 2.0 * w * _s_int(t)
        Mp = Mp + dg * _s(t)
        Mpp = Mpp + dg * _s_d(t) / (2.0 * w)
    return M, Mp, Mpp


def eps_from_M(M, Mp, Mpp):
    n = 1.0 + 1e-6 * M
    return n * n, 2.0 * n * 1e-6 * Mp, 2e-12 * Mp * Mp + 2.0 * n * 1e-6 * Mpp


def f_trilinear_duct(z_t, g_d, M0=330.0, g_std=0.118, w=1.0, wg=1.0):
    """Surface duct: M slope g_std on [0, z_t/3), g_d on [z_t/3, z_t), g_std
    above; kinks rounded over +-w; even quartic continuation below wg."""
    z_b = z_t / 3.0
    kinks = [(z_b, g_d - g_std), (z_t, g_std - g_d)]
    assert z_b - w > wg

    def Mfun(z):
        return modified_refractivity(z, M0, g_std, kinks, w)

    # even quartic below wg (M'' = 0 at wg for these parameters, kept general)
    Mw, Mpw, Mppw = (v[0] for v in Mfun(np.array([wg])))
    c4 = (Mppw - Mpw / wg) / (8.0 * wg * wg)
    c2 = (Mpw / wg - 4.0 * c4 * wg * wg) / 2.0
    c0 = Mw - c2 * wg ** 2 - c4 * wg ** 4

    def f(z):
        M, Mp, Mpp = Mfun(z)
        low = np.abs(z) < wg
        zl = z[low]
        M = M.copy(); Mp = Mp.copy(); Mpp = Mpp.copy()
        M[low] = c0 + c2 * zl ** 2 + c4 * zl ** 4
        Mp[low] = 2.0 * c2 * zl + 4.0 * c4 * zl ** 3
        Mpp[low] = 2.0 * c2 + 12.0 * c4 * zl ** 2
        return eps_from_M(M, Mp, Mpp)
    return f


def f_evaporation_duct(delta, M0=330.0, c1=0.125, z_rough=1.5e-4, zg=0.5):
    """Evaporation duct of height delta (log-linear M profile with roughness
    z_rough), continued below zg by the even quartic matching M, M', M'' there
    so that the reflected profile is C^2 at the ground."""
    def Mfun(z):
        zz = np.maximum(z, zg)
        M = M0 + c1 * zz - c1 * delta * np.log((zz + z_rough) / z_rough)
        Mp = c1 - c1 * delta / (zz + z_rough)
        Mpp = c1 * delta / (zz + z_rough) ** 2
        return M, Mp, Mpp

    Mw, Mpw, Mppw = (v[0] for v in Mfun(np.array([zg])))
    c4 = (Mppw - Mpw / zg) / (8.0 * zg * zg)
    c2 = (Mpw / zg - 4.0 * c4 * zg * zg) / 2.0
    c0 = Mw - c2 * zg ** 2 - c4 * zg ** 4

    def f(z):
        M, Mp, Mpp = Mfun(z)
        low = np.abs(z) < zg
        zl = z[low]
        M = M.copy(); Mp = Mp.copy(); Mpp = Mpp.copy()
        M[low] = c0 + c2 * zl ** 2 + c4 * zl ** 4
        Mp[low] = 2.0 * c2 * zl + 4.0 * c4 * zl ** 3
        Mpp[low] = 2.0 * c2 + 12.0 * c4 * zl ** 2
        return eps_from_M(M, Mp, Mpp)
    return f


# ----------------------------------------------------------------------------
# incident fields
# ----------------------------------------------------------------------------

def gaussian_beam(z, k, z_c, w0, tilt_rad):
    """exp(-((z-z_c)/w0)^2) exp(i k sin(tilt) (z - z_c)); w0 = 1/e radius."""
    y = z - z_c
    return np.exp(-(y / w0) ** 2) * np.exp(1j * k * math.sin(tilt_rad) * y)


def antenna_beam(z, k, z_s, theta_bw_rad, bc):
    """Gaussian antenna of half-power full beamwidth theta_bw at height z_s,
    elevation 0: angular spectrum exp(-ln2 kappa^2 / (2 sin^2(theta_bw/2))),
    unit peak, plus the ground image (+ Neumann, - Dirichlet)."""
    a = (k * math.sin(theta_bw_rad / 2.0)) ** 2 / (2.0 * math.log(2.0))
    u = np.exp(-a * (z - z_s) ** 2)
    if bc == BC_NEUMANN:
        u = u + np.exp(-a * (z + z_s) ** 2)
    elif bc == BC_DIRICHLET:
        u = u - np.exp(-a * (z + z_s) ** 2)
    return u.astype(np.complex128)


# ----------------------------------------------------------------------------
# workloads
# ----------------------------------------------------------------------------

def config_unit_periodic(n_screens=10):
    """Unit wavelength (k = 2 pi), 200 lambda x 64 lambda, N_z = 512, 10
    screens of 20 lambda.  eps = 1 for x < 100, eps = 1 + 1e-3 z beyond; the
    jump sits on screen edge q = 5.  Tilted (+2 deg) Gaussian beam of waist
    4 lambda at z = 32.  Periodic in z, no absorber, theta_max = 30 deg,
    a ray per grid point, 8 RK4 steps per screen."""
    k = 2.0 * math.pi
    z0, dzp = -48.0, 0.125
    n_p = int(round((112.0 - z0) / dzp)) + 1
    prof = _table([0.0, 100.0, 100.0, 200.0], z0, dzp, n_p,
                  [f_const(1.0), f_const(1.0), f_linear(1.0, 1e-3), f_linear(1.0, 1e-3)])
    n_z = 512
    z = 64.0 / n_z * np.arange(n_z)
    u0 = gaussian_beam(z, k, 32.0, 4.0, math.radians(2.0))
    return Problem("unit-periodic-512", k, 0.0, 64.0, n_z, BC_PERIODIC, 0.0, 20.0,
                   n_screens, prof, u0, math.radians(30.0), 1, 8, 0.0)


def config_homogeneous(eps0=1.0, n_z=256, height=32.0, dx=15.0, n_screens=3,
                       theta_deg=30.0, ray_stride=1, rk4_steps=4, bc=BC_PERIODIC,
                       tilt_deg=5.0):
    """Homogeneous medium eps = eps0 (closed-form angular-spectrum case)."""
    k = 2.0 * math.pi
    L = height * (2 if bc != BC_PERIODIC else 1)
    z0, dzp = -2.0 * L - dx, 0.125
    n_p = int(round((4.0 * L + 2 * dx) / dzp)) + 1
    prof = _table([0.0], z0, dzp, n_p, [f_const(eps0)])
    z = height / n_z * np.arange(n_z)
    if bc == BC_PERIODIC:
        u0 = gaussian_beam(z, k, height / 2, 3.0, math.radians(tilt_deg))
    else:
        prof = _table([0.0], 0.0, dzp, int(round((L + 2 * dx) / dzp)) + 1, [f_const(eps0)])
        u0 = antenna_beam(z, k, height / 3, math.radians(8.0), bc)
    return Problem(f"homogeneous-{n_z}", k, 0.0, height, n_z, bc, 0.0, dx, n_screens,
                   prof, u0, math.radians(theta_deg), ray_stride, rk4_steps, 0.0)


def config_gaussian_medium(a=0.02, b=0.01, n_z=256, height=64.0, dx=10.0, n_screens=3,
                           ray_stride=2, rk4_steps=8, theta_deg=20.0, seed=0):
    """Paper's exponential permittivity eps = 1 + a exp(-b (z - H/2)^2),
    periodic, with a tilted Gaussian beam (k = 2 pi)."""
    rng = np.random.default_rng(seed)
    k = 2.0 * math.pi
    zc = height / 2
    z0, dzp = -height, 0.0625
    n_p = int(round(3 * height / dzp)) + 1
    prof = _table([0.0], z0, dzp, n_p, [f_gaussian(a, b, zc=zc)])
    z = height / n_z * np.arange(n_z)
    tilt = float(rng.uniform(-3.0, 3.0))
    u0 = gaussian_beam(z, k, zc + float(rng.uniform(-4, 4)), 4.0, math.radians(tilt))
    return Problem(f"gaussian-medium-{n_z}", k, 0.0, height, n_z, BC_PERIODIC, 0.0, dx,
                   n_screens, prof, u0, math.radians(theta_deg), ray_stride, rk4_steps, 0.0,
                   meta={"tilt_deg": tilt})


def config_gaussian_layer(a, b, height, n_z, range_m, n_screens, n_max, lam=0.05, w0=60.0,
                          tilt_deg=0.0, ray_stride=16, rk4_steps=16):
    """Periodic domain [-height/2, height/2) around a Gaussian permittivity
    layer eps = 1 + a exp(-b z^2) (the paper's exponential model, centred),
    x-invariant; Gaussian beam of waist w0 at z = 0, tilted by tilt_deg;
    n_max fixes the kept modes."""
    k = 2.0 * math.pi / lam
    dx = range_m / n_screens
    z0 = -height / 2 - 2.0 * dx * 0.05 - 8.0
    dzp = 0.05
    n_p = int(math.ceil((height + 2.0 * (-height / 2 - z0)) / dzp)) + 1
    prof = _table([0.0], z0, dzp, n_p, [f_gaussian(a, b)])
    z = -height / 2 + height / n_z * np.arange(n_z)
    u0 = gaussian_beam(z, k, 0.0, w0, math.radians(tilt_deg))
    return Problem(f"gaussian-layer-{n_z}", k, -height / 2, height / 2, n_z, BC_PERIODIC, 0.0,
                   dx, n_screens, prof, u0, math.radians(89.0), ray_stride, rk4_steps, 0.0,
                   n_max=n_max, meta={"a": a, "b": b})


def config_gaussian_lens_40km(**kw):
    """A single-focus lens like the paper's first example: eps = 1 + 1e-4
    exp(-1e-4 z^2), lambda = 5 cm, 401 modes, 40 km in 40 screens of 1 km,
    600 m periodic domain, 60 m beam (focus near 16 km)."""
    return config_gaussian_layer(1e-4, 1e-4, 600.0, 4096, 40_000.0, 40, 200, **kw)


def config_gaussian_duct_200km(**kw):
    """A narrow duct like the paper's second example: eps = 1 + 1e-4
    exp(-1e-3 z^2), lambda = 5 cm, beam tilted 0.2 deg, 200 km in 200 screens
    of 1 km (about ten oscillations in the duct), 400 m periodic domain, 241
    modes."""
    return config_gaussian_layer(1e-4, 1e-3, 400.0, 4096, 200_000.0, 200, 120, w0=10.0,
                                 tilt_deg=0.2, **kw)


def config_surface_duct(seed=2, height=200.0, n_z=16384, range_m=10_000.0, n_screens=200,
                        lam=0.05, theta_bw_deg=1.0, z_s=10.0, z_t_range=(20.0, 60.0),
                        g_d_range=(-0.2, -0.05), theta_max_deg=3.5, ray_stride=16,
                        rk4_steps=16, bc=BC_NEUMANN, absorber_frac=0.2, dzp=0.05):
    """Surface duct over a reflecting ground: lambda = 5 cm, height 200 m,
    N_z = 16384, 10 km in 200 screens.  Trilinear M(z) with duct top z_t ~
    U(20, 60) m and trapping-layer gradient g_d ~ U(-0.2, -0.05) M/m (seeded),
    Gaussian antenna of 1 deg beamwidth at 10 m, Neumann ground, top absorber
    over the upper 20 % of the height."""
    rng = np.random.default_rng(seed)
    z_t = float(rng.uniform(*z_t_range))
    g_d = float(rng.uniform(*g_d_range))
    k = 2.0 * math.pi / lam
    dx = range_m / n_screens
    top = height + 2.0 * dx * math.tan(math.radians(theta_max_deg)) + 8.0
    n_p = int(math.ceil(top / dzp)) + 1
    prof = _table([0.0], 0.0, dzp, n_p, [f_trilinear_duct(z_t, g_d)])
    z = height / n_z * np.arange(n_z)
    u0 = antenna_beam(z, k, z_s, math.radians(theta_bw_deg), bc)
    return Problem(f"surface-duct-{n_z}", k, 0.0, height, n_z, bc, 0.0, dx, n_screens,
                   prof, u0, math.radians(theta_max_deg), ray_stride, rk4_steps,
                   absorber_frac, meta={"z_t": z_t, "g_d": g_d, "seed": seed})


def config_surface_duct_small(seed=12, n_screens=6, n_z=4096, height=50.0, **kw):
    """Same physics as the 200 m duct at the same grid spacing, 50 m high
    (duct top U(10, 20) m, antenna at 5 m), sized for the CPU oracle."""
    return config_surface_duct(seed=seed, height=height, n_z=n_z,
                               range_m=50.0 * n_screens, n_screens=n_screens,
                               z_s=5.0, z_t_range=(10.0, 20.0), **kw)


def config_range_dependent_duct(seed=3, height=500.0, n_z=131072, range_m=100_000.0,
                                n_screens=2000, lam=0.05, theta_bw_deg=0.5, z_s=25.0,
                                theta_max_deg=2.0, ray_stride=64, rk4_steps=16,
                                col_every_m=1000.0, dzp=0.05):
    """Paper-scale duct: 500 m high, N_z = 131072, 100 km in 2000 screens; the
    duct top varies linearly by +-30 % over the range (sign seeded), with a
    column of the table every col_every_m metres."""
    rng = np.random.default_rng(seed)
    z_t0 = float(rng.uniform(20.0, 60.0))
    g_d = float(rng.uniform(-0.2, -0.05))
    sgn = 1.0 if rng.uniform() < 0.5 else -1.0
    k = 2.0 * math.pi / lam
    dx = range_m / n_screens
    top = height + 2.0 * dx * math.tan(math.radians(theta_max_deg)) + 8.0
    n_p = int(math.ceil(top / dzp)) + 1
    n_cols = int(round(range_m / col_every_m)) + 1
    xs = np.linspace(0.0, range_m, n_cols)
    cols = [f_trilinear_duct(z_t0 * (1.0 + 0.3 * sgn * (2.0 * x / range_m - 1.0)), g_d) for x in xs]
    prof = _table(xs, 0.0, dzp, n_p, cols)
    z = height / n_z * np.arange(n_z)
    u0 = antenna_beam(z, k, z_s, math.radians(theta_bw_deg), BC_NEUMANN)
    return Problem(f"range-dependent-duct-{n_z}", k, 0.0, height, n_z, BC_NEUMANN, 0.0, dx,
                   n_screens, prof, u0, math.radians(theta_max_deg), ray_stride, rk4_steps,
                   0.2, meta={"z_t0": z_t0, "g_d": g_d, "sign": sgn, "seed": seed})


def config_open_lens(n_z=131072, fc_patch=920, fc_overlap=224, seed=5, n_screens=100,
                     dx=5.0, n_beams=8, a=0.002, theta_max_deg=60.0, ray_stride=8,
                     rk4_steps=8, dzp=0.0625):
    """Open (non-periodic) interval for the patch-wise continuation method:
    unit wavelength, three grid points per wavelength (N_z = 131072: 43 690
    wavelengths, 188 patches of 920 points sharing 224), a broad Gaussian
    lens eps = 1 + a exp(-((z - H/2) / (H/6))^2), and n_beams seeded Gaussian
    beams (waists 3-10 wavelengths, tilts within +-20 deg) in the middle 70 %
    of the interval, so that the field vanishes near both ends over the
    range; screens of dx = 5 wavelengths."""
    rng = np.random.default_rng(seed)
    k = 2.0 * math.pi
    h = 1.0 / 3.0
    H = n_z * h
    # launch ghosts and the rays' reach beyond both ends
    margin = 3.0 * dx * math.tan(math.radians(theta_max_deg)) + 6.0 * ray_stride * h + 4.0
    z0 = -margin
    n_p = int(math.ceil((H + 2.0 * margin) / dzp)) + 1
    zc, wl = H / 2, H / 6

    def lens(z):
        y = (z - zc) / wl
        g = a * np.exp(-y * y)
        return 1.0 + g, -2.0 * y / wl * g, (4.0 * y * y - 2.0) / (wl * wl) * g
    prof = _table([0.0], z0, dzp, n_p, [lens])
    z = h * np.arange(n_z)
    u0 = np.zeros(n_z, dtype=np.complex128)
    for _ in range(n_beams):
        c = float(rng.uniform(0.15, 0.85)) * H
        u0 += gaussian_beam(z, k, c, float(rng.uniform(3.0, 10.0)),
                            math.radians(float(rng.uniform(-20.0, 20.0))))
    return Problem(f"open-lens-{n_z}", k, 0.0, H, n_z, BC_OPEN, 0.0, dx, n_screens, prof, u0,
                   math.radians(theta_max_deg), ray_stride, rk4_steps, 0.0,
                   fc_patch=fc_patch, fc_overlap=fc_overlap, meta={"seed": seed, "a": a})


def random_request(rng, n_z_range=(1 << 12, 1 << 16), range_km=(5.0, 50.0), screens_per_km=20,
                   dzp=0.05):
    """One instance of the uneven batch / served stream: frequency U(1, 10)
    GHz, height U(100, 400) m, N_z = 2^ceil(log2(4 H / lambda)) clamped to
    n_z_range, range U(range_km) at screens_per_km, trilinear or evaporation
    duct (coin flip; duct top U(20, 60) m and gradient U(-0.2, -0.05) M/m, or
    evaporation height U(5, 40) m), Gaussian antenna of beamwidth U(0.5, 2) deg
    at U(5, 30) m, theta_max = 3 beamwidths + 0.5 deg, one ray per R grid
    points with R the power of two nearest 0.25 m / dz, 16 RK4 steps."""
    f_hz = float(rng.uniform(1e9, 10e9))
    lam = 299_792_458.0 / f_hz
    H = float(rng.uniform(100.0, 400.0))
    n_z = int(2 ** math.ceil(math.log2(4.0 * H / lam)))
    n_z = int(min(max(n_z, n_z_range[0]), n_z_range[1]))
    rng_m = float(rng.uniform(*range_km)) * 1000.0
    n_screens = max(1, int(round(rng_m / 1000.0 * screens_per_km)))
    dx = 1000.0 / screens_per_km
    bw = float(rng.uniform(0.5, 2.0))
    z_s = float(rng.uniform(5.0, 30.0))
    theta_max = math.radians(3.0 * bw + 0.5)
    dz = H / n_z
    R = int(2 ** round(math.log2(max(0.25 / dz, 1.0))))
    k = 2.0 * math.pi / lam
    if rng.uniform() < 0.5:
        prof_f = f_trilinear_duct(float(rng.uniform(20.0, 60.0)), float(rng.uniform(-0.2, -0.05)))
        kind = "trilinear"
    else:
        prof_f = f_evaporation_duct(float(rng.uniform(5.0, 40.0)))
        kind = "evaporation"
    top = H + 2.0 * dx * math.tan(theta_max) + 8.0 + 2 * R * dz * (
        math.ceil(dx * math.tan(theta_max) / (R * dz)) + 4)
    n_p = int(math.ceil(top / dzp)) + 1
    prof = _table([0.0], 0.0, dzp, n_p, [prof_f])
    z = H / n_z * np.arange(n_z)
    u0 = antenna_beam(z, k, z_s, math.radians(bw), BC_NEUMANN)
    return Problem(f"request-{kind}-{n_z}", k, 0.0, H, n_z, BC_NEUMANN, 0.0, dx, n_screens,
                   prof, u0, theta_max, R, 16, 0.2,
                   meta={"f_hz": f_hz, "range_m": n_screens * dx, "profile": kind,
                         "beamwidth_deg": bw, "z_s": z_s})


def batch_uneven(seed=4, n=64, **kw):
    """64 uneven instances (frequency, height, N_z, range, duct profile)."""
    rng = np.random.default_rng(seed)
    return [random_request(rng, **kw) for _ in range(n)]


class HillInputs:
    """Inputs of one separation-of-variables problem batch: the boundary
    condition and domain, K modes, eps sampled at n_q + 1 points of the half
    period from the symmetry point z_c, wavenumbers, fields at x = 0 and the
    output ranges."""

    def __init__(self, name, bc, z_a, z_b, z_c, K, eps_half, k, u0, xs):
        self.name, self.bc, self.z_a, self.z_b, self.z_c = name, bc, z_a, z_b, z_c
        self.K = K
        self.eps = np.atleast_2d(np.asarray(eps_half, float))
        self.k = np.atleast_1d(np.asarray(k, float))
        self.u0 = np.atleast_2d(np.asarray(u0, complex))
        self.xs = np.atleast_1d(np.asarray(xs, float))
        self.n_q = self.eps.shape[1] - 1
        self.n_z = self.u0.shape[1]


def hill_surface_duct_2km(K=640, n_q=1 << 15, batch=1):
    """The 16384-point surface duct (200 m, Neumann ground, no absorber) as a
    separation-of-variables problem at 2 km; batch > 1 adds ducts of seeds
    3, 4, ... (own duct top and gradient) at the same wavenumber."""
    epss, u0s, ks = [], [], []
    for b in range(batch):
        pb = config_surface_duct(seed=2 + b, n_screens=40, range_m=2000.0)
        f = f_trilinear_duct(pb.meta["z_t"], pb.meta["g_d"])
        s = (pb.z_b - pb.z_a) * np.arange(n_q + 1) / n_q
        epss.append(f(s)[0])
        u0s.append(pb.u0)
        ks.append(pb.k)
    return HillInputs(f"hill-surface-duct-16384-K{K}", BC_NEUMANN, pb.z_a, pb.z_b, pb.z_a, K,
                      epss, ks, u0s, [2000.0])


def hill_gaussian_duct_200km(n_q=4096, extra_modes=100):
    """The 400 m periodic domain with the narrow Gaussian duct at its centre
    (eps = 1 + 1e-4 exp(-1e-3 z^2), lambda = 5 cm, 0.2 deg beam), 200 km,
    K = n_max + extra_modes, eps even about z_c = 0."""
    pb = config_gaussian_duct_200km()
    L = pb.z_b - pb.z_a
    s = np.arange(n_q + 1) * L / (2 * n_q)
    eps = f_gaussian(pb.meta["a"], pb.meta["b"])(s)[0]
    return HillInputs("hill-gaussian-duct-200km", BC_PERIODIC, pb.z_a, pb.z_b, 0.0,
                      pb.n_max + extra_modes, eps, pb.k, pb.u0, [200_000.0])


def hill_gaussian_lens_40km(n_q=4096, extra_modes=100):
    """The 600 m periodic domain with the single-focus Gaussian lens at its
    centre (eps = 1 + 1e-4 exp(-1e-4 z^2), lambda = 5 cm, 60 m beam), 40 km,
    K = n_max + extra_modes, eps even about z_c = 0."""
    pb = config_gaussian_lens_40km()
    L = pb.z_b - pb.z_a
    s = np.arange(n_q + 1) * L / (2 * n_q)
    eps = f_gaussian(pb.meta["a"], pb.meta["b"])(s)[0]
    return HillInputs("hill-gaussian-lens-40km", BC_PERIODIC, pb.z_a, pb.z_b, 0.0,
                      pb.n_max + extra_modes, eps, pb.k, pb.u0, [40_000.0])


WORKLOADS = {
    "unit-periodic-512": config_unit_periodic,
    "surface-duct-16384": config_surface_duct,
    "surface-duct-small-4096": config_surface_duct_small,
    "range-dependent-duct-131072": config_range_dependent_duct,
}
