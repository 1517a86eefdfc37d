"""Plain, slow FP64 CPU oracle of the screened-WKB (S-WKB) method.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  The CUDA library never calls it and
shares no code with it: the two meet only in the seeded inputs of
paper_2301_03814_gb300.workloads (tables and fields, no method arithmetic).

What it computes (Bruno & Maas, "WKB Across Caustics: The Screened-WKB
Method"), per screen Gamma_q -> Gamma_{q+1}, in the order of Algorithm 1:

  (a) vertical DFT of the screen field (Eq. fft_eq / ifft_eq), keeping the
      plane-wave modes |n| <= n_max (the rest are evanescent or filtered);
  (b) for every kept mode, rays launched with the initial conditions of
      Sec. 2.1.2 (psi_z = kappa_n, psi_x = sqrt(eps - kappa_n^2), A = w_n/N)
      and integrated across the slab with classical RK4 on the characteristic
      system (Eq. charsys) and its s-variation (Eq. charsys_s), written with x
      as the ray parameter; the amplitude comes from the ray-tube Jacobian
      (Eqs. delta_psi_eq, delta_psi_eq_jac, transport_xt) in its corrected form
      A = A0 sqrt(J(s,0)/J(s,t)) = A0 sqrt(P0 / (P1 Z_s));
  (c) 4-point Lagrange interpolation of each mode's phase and amplitude from
      the ray landing points onto the grid of Gamma_{q+1} (Eq.
      ray_bundle_q_plus_1);
  (d) the sum over modes (Eq. ray_bundle_q_plus_1 / Algorithm 1, last step).

Readings of the paper taken here where it is garbled or silent (each one is
also implemented, separately, by the CUDA library):

  R1  the DFT is the standard one on the grid z_m = z_lo + m dz, m = 0..N-1:
      w_n = sum_m u_m exp(-2 pi i n m / N), u_m = (1/N) sum_n w_n e^{ik psi_n}.
  R2  psi_n(x_q, z) = kappa_n (z - z_lo), kappa_n = 2 pi n / (k L).
  R4  modes with |n| > n_max = floor(sin(theta_max) L / lambda) are dropped.
  R5  rays are parametrised by x (d/dx = (1/2P) d/dt); P comes from the
      eikonal P = sqrt(eps - Q^2), so only eps, eps_z, eps_zz are needed.  The
      integrator is classical RK4 with N_t equal steps per screen.
  R6  J = X_t Z_s - Z_t X_s (sign typo in the paper), Delta psi = J_t / (2 J)
      (the paper drops the 2), hence A = A0 sqrt(J0 / J); with x as parameter
      J = 2 P Z_s|_x and J0 = 2 P0.
  R7  any Z_s <= 0 (a caustic between screens, Remark after Eq.
      ray_bundle_q_plus_1) or eps - Q^2 <= 0 (a turning point in x) is an
      error, never silently continued.
  R8  rays every R grid points plus G ghost rays on each side,
      G = ceil(dx tan(theta) / (R dz)) + 3, tan(theta) of the steepest kept
      mode; bracket j of grid point m has delta_j <= m < delta_{j+1} in grid
      units; stencil j-1..j+2.
  R9  Neumann / Dirichlet ground at z_a by reflection (Sec. 2.3): the period is
      [2 z_a - z_b, z_b), eps~(z) = eps(z_a + |z - z_a|), and after every
      screen the field is projected onto even / odd functions,
      u <- (u(z) +- u(2 z_a - z)) / 2.  An optional top absorber multiplies the
      field by cos^2(pi/2 (|z - z_a| - (1-f) H) / (f H)) above (1-f) H.
  R10 eps is evaluated from its table by quintic Hermite interpolation in z
      (C^2) and linear interpolation in x between the columns bracketing x;
      at the start of a screen the right limit in x is used, at its end the
      left limit.
  R15 fields between screens (Sec. 2.1, the remark that extra interpolation
      points may be added for visualisation): on the planes x_q + j dx / P,
      j = 1..P with P dividing N_t (RK4 step boundaries), the screen's modes
      and rays marched j N_t / P steps, interpolated and summed exactly as on
      the screen; the absorber is a screen-level device and multiplies only
      the screen's own field (j = P); grounded fields are projected onto
      even / odd functions like screen fields.

Everything is float64.  Functions raise OracleError subclasses on R7 events.
"""
from __future__ import annotations

import math
from dataclasses import dataclass

import numpy as np

PERIODIC, NEUMANN, DIRICHLET = 0, 1, 2


class OracleError(RuntimeError):
    code = "error"


class CausticError(OracleError):
    code = "caustic"


class TurningError(OracleError):
    code = "turning"


class RangeError(OracleError):
    code = "range"


# ----------------------------------------------------------------------------
# medium: quintic Hermite in z, linear in x (reading R10)
# ----------------------------------------------------------------------------

def hermite5(f0, d0, s0, f1, d1, s1, t, h):
    """Quintic Hermite interpolant on one interval of length h at local
    coordinate t in [0, 1], from value / first / second derivative at both
    ends.  Returns value, d/dz, d2/dz2.  Basis written out term by term."""
    t2 = t * t
    t3 = t2 * t
    t4 = t3 * t
    t5 = t4 * t
    # basis functions and their t-derivatives
    H0 = 1 - 10 * t3 + 15 * t4 - 6 * t5
    H1 = t - 6 * t3 + 8 * t4 - 3 * t5
    H2 = 0.5 * t2 - 1.5 * t3 + 1.5 * t4 - 0.5 * t5
    H3 = 10 * t3 - 15 * t4 + 6 * t5
    H4 = -4 * t3 + 7 * t4 - 3 * t5
    H5 = 0.5 * t3 - t4 + 0.5 * t5
    dH0 = -30 * t2 + 60 * t3 - 30 * t4
    dH1 = 1 - 18 * t2 + 32 * t3 - 15 * t4
    dH2 = t - 4.5 * t2 + 6 * t3 - 2.5 * t4
    dH3 = 30 * t2 - 60 * t3 + 30 * t4
    dH4 = -12 * t2 + 28 * t3 - 15 * t4
    dH5 = 1.5 * t2 - 4 * t3 + 2.5 * t4
    ddH0 = -60 * t + 180 * t2 - 120 * t3
    ddH1 = -36 * t + 96 * t2 - 60 * t3
    ddH2 = 1 - 9 * t + 18 * t2 - 10 * t3
    ddH3 = 60 * t - 180 * t2 + 120 * t3
    ddH4 = -24 * t + 84 * t2 - 60 * t3
    ddH5 = 3 * t - 12 * t2 + 10 * t3
    v = f0 * H0 + h * d0 * H1 + h * h * s0 * H2 + f1 * H3 + h * d1 * H4 + h * h * s1 * H5
    dv = (f0 * dH0 + h * d0 * dH1 + h * h * s0 * dH2 + f1 * dH3 + h * d1 * dH4 + h * h * s1 * dH5) / h
    ddv = (f0 * ddH0 + h * d0 * ddH1 + h * h * s0 * ddH2 + f1 * ddH3 + h * d1 * ddH4
           + h * h * s1 * ddH5) / (h * h)
    return v, dv, ddv


class Medium:
    """eps(x, z) with eps_z and eps_zz from a profile table (R10, R9)."""

    def __init__(self, profile, mirrored: bool, z_mirror: float):
        self.x_cols = np.asarray(profile.x_cols, dtype=np.float64)
        self.z0 = float(profile.z0)
        self.dz = float(profile.dz)
        self.e = np.asarray(profile.eps, dtype=np.float64)
        self.ez = np.asarray(profile.eps_z, dtype=np.float64)
        self.ezz = np.asarray(profile.eps_zz, dtype=np.float64)
        self.n_p = self.e.shape[1]
        self.mirrored = mirrored
        self.z_mirror = z_mirror

    def column_weights(self, x: float, right: bool):
        """Columns (c, c+1) and weight theta of c+1 for range x.  right=True
        takes the right limit at a column position, right=False the left."""
        n = len(self.x_cols)
        if n == 1:
            return 0, 0.0
        if right:
            c = int(np.sum(self.x_cols <= x)) - 1
        else:
            c = int(np.sum(self.x_cols < x)) - 1
        c = min(max(c, 0), n - 2)
        span = self.x_cols[c + 1] - self.x_cols[c]
        th = 0.0 if span <= 0 else (x - self.x_cols[c]) / span
        return c, min(max(th, 0.0), 1.0)

    def column_eval(self, c: int, z: np.ndarray):
        u = (z - self.z0) / self.dz
        if np.any(u < 0) or np.any(u > self.n_p - 1):
            raise RangeError("ray left the permittivity table")
        i = np.minimum(np.floor(u).astype(np.int64), self.n_p - 2)
        t = u - i
        e, ez, ezz = self.e[c], self.ez[c], self.ezz[c]
        return hermite5(e[i], ez[i], ezz[i], e[i + 1], ez[i + 1], ezz[i + 1], t, self.dz)

    def eval(self, x: float, right: bool, z: np.ndarray):
        if self.mirrored:
            sgn = np.where(z < self.z_mirror, -1.0, 1.0)
            zz = self.z_mirror + np.abs(z - self.z_mirror)
        else:
            sgn = 1.0
            zz = z
        c, th = self.column_weights(x, right)
        if th == 0.0:
            e, ez, ezz = self.column_eval(c, zz)
        elif th == 1.0:
            e, ez, ezz = self.column_eval(c + 1, zz)
        else:
            a = self.column_eval(c, zz)
            b = self.column_eval(c + 1, zz)
            e, ez, ezz = ((1.0 - th) * a[i] + th * b[i] for i in range(3))
        return e, sgn * ez, ezz


# ----------------------------------------------------------------------------
# plan-level derived quantities
# ----------------------------------------------------------------------------

@dataclass
class Geometry:
    N: int          # FFT length (period points)
    L: float        # period length
    dz: float       # grid spacing
    z_lo: float     # first grid point of the period
    n_max: int
    M: int
    R: int
    N_r: int        # rays per mode without ghosts
    G: int          # ghost rays per side
    NRT: int        # rays per mode with ghosts
    mirrored: bool


def geometry(pb) -> Geometry:
    """Grid, mode set (R4) and ray layout (R8) of a workloads.Problem."""
    mirrored = pb.bc != PERIODIC
    H = pb.z_b - pb.z_a
    N = pb.n_z * (2 if mirrored else 1)
    L = H * (2 if mirrored else 1)
    dz = H / pb.n_z
    z_lo = pb.z_a - H if mirrored else pb.z_a
    lam = 2.0 * math.pi / pb.k
    if pb.n_max > 0:
        n_max = int(pb.n_max)
    else:
        n_max = int(math.floor(math.sin(pb.theta_max) * L / lam * (1.0 + 1e-12)))
    n_max = min(n_max, N // 2 - 1)
    R = int(pb.ray_stride)
    if N % R:
        raise ValueError("ray stride must divide the FFT length")
    N_r = N // R
    kmax = n_max * lam / L
    tan_t = kmax / math.sqrt(1.0 - kmax * kmax)
    G = int(math.ceil(pb.dx * tan_t / (R * dz) - 1e-9)) + 3
    return Geometry(N, L, dz, z_lo, n_max, 2 * n_max + 1, R, N_r, G, N_r + 2 * G, mirrored)


def absorber(pb, g: Geometry) -> np.ndarray:
    """Top absorber window W(z_m) (R9); ones when absorber_frac == 0."""
    W = np.ones(g.N)
    f = pb.absorber_frac
    if f <= 0:
        return W
    H = pb.z_b - pb.z_a
    z = g.z_lo + g.dz * np.arange(g.N)
    d = np.abs(z - pb.z_a) if g.mirrored else (z - pb.z_a)
    top = d > (1.0 - f) * H
    W[top] = np.cos(0.5 * math.pi * (d[top] - (1.0 - f) * H) / (f * H)) ** 2
    return W


# ----------------------------------------------------------------------------
# the propagator
# ----------------------------------------------------------------------------

class Oracle:
    def __init__(self, pb):
        self.pb = pb
        self.g = geometry(pb)
        self.medium = Medium(pb.profile, self.g.mirrored, pb.z_a)
        self.n = np.arange(-self.g.n_max, self.g.n_max + 1)
        self.kappa = 2.0 * math.pi * self.n / (pb.k * self.g.L)       # R2
        self.W = absorber(pb, self.g)
        self.sign = {PERIODIC: 0, NEUMANN: 1, DIRICHLET: -1}[pb.bc]

    # -- field layout on the full period -------------------------------------
    def extend(self, u_phys: np.ndarray) -> np.ndarray:
        """Physical field -> field on the whole period (mirror image for
        grounded domains; the point 2 z_a - z_b has no physical partner and is
        set to 0)."""
        g = self.g
        u_phys = np.asarray(u_phys, dtype=np.complex128)
        if not g.mirrored:
            return u_phys.copy()
        nz = self.pb.n_z
        u = np.zeros(g.N, dtype=np.complex128)
        u[nz:] = u_phys
        u[nz - np.arange(1, nz)] = self.sign * u_phys[1:]
        return u

    def project(self, u: np.ndarray) -> np.ndarray:
        """Reflection step (R9): u <- (u(z) +- u(2 z_a - z)) / 2."""
        if not self.g.mirrored:
            return u
        N = self.g.N
        mirror = u[(N - np.arange(N)) % N]
        return 0.5 * (u + self.sign * mirror)

    def restrict(self, u: np.ndarray) -> np.ndarray:
        if not self.g.mirrored:
            return u.copy()
        return u[self.pb.n_z:].copy()

    # -- step (a): DFT ----------------------------------------------------------
    def modes(self, u: np.ndarray) -> np.ndarray:
        """c_n = w_n / N for |n| <= n_max, w = DFT(u) (Eq. fft_eq, R1, R4)."""
        w = np.fft.fft(u)
        return w[self.n % self.g.N] / self.g.N

    # -- step (b): rays -----------------------------------------------------------
    def stage_x(self, q: int):
        """RK4 stage positions of screen q: (x, right-limit?) for l = 0..2N_t
        (l/2 steps in); the last one is the next screen, taken from the left."""
        pb = self.pb
        x_q = pb.x0 + q * pb.dx
        x_next = pb.x0 + (q + 1) * pb.dx
        h = pb.dx / pb.rk4_steps
        out = [(x_q + 0.5 * l * h, True) for l in range(2 * pb.rk4_steps)]
        out.append((x_next, False))
        return out

    def rhs(self, xs, kappa, z, Q, r, Zs, Qs):
        """x-form of Eqs. charsys / charsys_s (R5):
        z' = Q/P, Q' = eps_z/(2P), r' = (eps - kappa Q)/P  with r = psi - kappa (z - z_lo),
        P_s = (eps_z Z_s - 2 Q Q_s)/(2P), Z_s' = (Q_s - Q P_s / P)/P,
        Q_s' = eps_zz Z_s/(2P) - eps_z P_s/(2P^2)."""
        x, right = xs
        e, ez, ezz = self.medium.eval(x, right, z)
        P2 = e - Q * Q
        if np.any(P2 <= 0.0):
            raise TurningError("eps - Q^2 <= 0 on a ray")
        if np.any(Zs <= 0.0):
            raise CausticError("Z_s <= 0: caustic between screens")
        P = np.sqrt(P2)
        dz = Q / P
        dQ = ez / (2.0 * P)
        dr = (e - kappa * Q) / P
        Ps = (ez * Zs - 2.0 * Q * Qs) / (2.0 * P)
        dZs = (Qs - Q * Ps / P) / P
        dQs = ezz * Zs / (2.0 * P) - ez * Ps / (2.0 * P * P)
        return dz, dQ, dr, dZs, dQs

    def march(self, q: int, kappa: np.ndarray, s: np.ndarray, steps: int | None = None):
        """RK4 across screen q for rays (kappa, s) (arrays of one shape).
        Returns dict with landing z, Q, residual r, Z_s, Q_s, P0, P1 and the
        amplitude factor a = sqrt(P0 / (P1 Z_s)) (R6).  steps < rk4_steps
        stops on the plane x_q + steps h inside the screen (R15), with P1
        evaluated there."""
        pb = self.pb
        n_steps = pb.rk4_steps if steps is None else int(steps)
        xs = self.stage_x(q)
        h = pb.dx / pb.rk4_steps
        kappa, s = np.broadcast_arrays(np.asarray(kappa, dtype=np.float64),
                                       np.asarray(s, dtype=np.float64))
        z = s.copy()
        Q = kappa.copy()
        kap = Q.copy()
        r = np.zeros_like(z)
        Zs = np.ones_like(z)
        Qs = np.zeros_like(z)
        e0, _, _ = self.medium.eval(xs[0][0], xs[0][1], z)
        P0sq = e0 - kap * kap
        if np.any(P0sq <= 0):
            raise TurningError("mode is evanescent at launch")
        P0 = np.sqrt(P0sq)
        y = (z, Q, r, Zs, Qs)
        for i in range(n_steps):
            a = xs[2 * i]
            m = xs[2 * i + 1]
            b = xs[2 * i + 2]
            k1 = self.rhs(a, kap, *y)
            k2 = self.rhs(m, kap, *(yi + 0.5 * h * ki for yi, ki in zip(y, k1)))
            k3 = self.rhs(m, kap, *(yi + 0.5 * h * ki for yi, ki in zip(y, k2)))
            k4 = self.rhs(b, kap, *(yi + h * ki for yi, ki in zip(y, k3)))
            y = tuple(yi + h / 6.0 * (p1 + 2.0 * p2 + 2.0 * p3 + p4)
                      for yi, p1, p2, p3, p4 in zip(y, k1, k2, k3, k4))
        z, Q, r, Zs, Qs = y
        if np.any(Zs <= 0.0):
            raise CausticError("Z_s <= 0 at landing")
        e1, _, _ = self.medium.eval(xs[2 * n_steps][0], xs[2 * n_steps][1], z)
        P1sq = e1 - Q * Q
        if np.any(P1sq <= 0):
            raise TurningError("eps - Q^2 <= 0 at landing")
        P1 = np.sqrt(P1sq)
        return dict(z=z, Q=Q, r=r, Zs=Zs, Qs=Qs, P0=P0, P1=P1, a=np.sqrt(P0 / (P1 * Zs)))

    def launch_points(self) -> np.ndarray:
        g = self.g
        j = np.arange(g.NRT)
        return g.z_lo + (j - g.G) * g.R * g.dz

    # -- step (c): interpolation --------------------------------------------------
    def interpolate(self, delta: np.ndarray, vals):
        """Values at grid points m = 0..N-1 from ray landings delta (grid
        units, increasing) by 4-point Lagrange on the bracket stencil (R8)."""
        g = self.g
        if np.any(np.diff(delta) <= 0):
            raise CausticError("ray landings not increasing (rays crossed)")
        m = np.arange(g.N, dtype=np.float64)
        j = np.searchsorted(delta, m, side="right") - 1
        if j.min() < 1 or j.max() > len(delta) - 3:
            raise RangeError("ghost rays do not cover the screen")
        x = [delta[j + o] for o in (-1, 0, 1, 2)]
        out = []
        for v in vals:
            f = [v[j + o] for o in (-1, 0, 1, 2)]
            acc = np.zeros(g.N)
            for p in range(4):
                wgt = np.ones(g.N)
                for l in range(4):
                    if l != p:
                        wgt = wgt * (m - x[l]) / (x[p] - x[l])
                acc = acc + wgt * f[p]
            out.append(acc)
        return out

    # -- one screen ------------------------------------------------------------------
    def screen(self, u: np.ndarray, q: int, keep_rays: bool = False):
        """Gamma_q -> Gamma_{q+1} on the full period (Algorithm 1)."""
        g = self.g
        pb = self.pb
        u = self.project(u)
        c = self.modes(u)                                            # (a)
        s = self.launch_points()
        rays = self.march(q, self.kappa[:, None], s[None, :])       # (b)
        out = self.modal_sum(c, rays) * self.W                       # (c) + (d)
        if keep_rays:
            return out, c, rays
        return out

    def modal_sum(self, c: np.ndarray, rays) -> np.ndarray:
        """Eq. ray_bundle_q_plus_1 on the grid: for every mode, phase and
        amplitude interpolated from its rays' landings (R8), then
        sum_n c_n A_n exp(i (k kappa_n (z_m - z_lo) + k r_n))."""
        g = self.g
        delta = (rays["z"] - g.z_lo) / g.dz
        out = np.zeros(g.N, dtype=np.complex128)
        for i in range(len(self.n)):
            out += self.mode_term(int(self.n[i]), c[i], delta[i], rays["r"][i], rays["a"][i])
        return out

    def mode_term(self, n: int, c_n: complex, delta: np.ndarray, r: np.ndarray,
                  a: np.ndarray) -> np.ndarray:
        """One mode's contribution to Eq. ray_bundle_q_plus_1 on the grid:
        phase and amplitude interpolated from the rays' landings delta (R8),
        c_n A_n(z_m) exp(i (k kappa_n (z_m - z_lo) + k r_n(z_m)))."""
        g = self.g
        m = np.arange(g.N)
        r_m, a_m = self.interpolate(delta, (r, a))
        base = 2.0 * math.pi * ((n * m) % g.N) / g.N                 # = k kappa_n (z_m - z_lo)
        return c_n * a_m * np.exp(1j * (base + self.pb.k * r_m))

    # -- fields between screens (Section 2: extra interpolation points) --------------
    def screen_planes(self, u: np.ndarray, q: int, planes: int):
        """Fields of screen q on the planes x_q + j dx / planes, j = 1..planes
        (R15): the screen's modes and rays, marched j rk4_steps / planes RK4
        steps, interpolated and summed like the screen itself.  The last plane
        is the screen's own field (absorber applied); the planes before it are
        the ray field between screens (no absorber)."""
        pb = self.pb
        if planes < 1 or pb.rk4_steps % planes:
            raise ValueError("planes must divide rk4_steps")
        u = self.project(u)
        c = self.modes(u)
        s = self.launch_points()
        out = []
        for j in range(1, planes + 1):
            rays = self.march(q, self.kappa[:, None], s[None, :],
                              steps=j * pb.rk4_steps // planes)
            f = self.modal_sum(c, rays)
            out.append(f * self.W if j == planes else f)
        return out

    def propagate_planes(self, u_phys: np.ndarray, q0: int, n_screens: int, planes: int):
        """Physical fields on every plane of screens q0 .. q0+n_screens-1,
        rows ordered (screen, plane); each screen starts from the previous
        screen's last plane."""
        u = self.extend(u_phys)
        rows = []
        for q in range(q0, q0 + n_screens):
            fields = self.screen_planes(u, q, planes)
            rows.extend(self.restrict(self.project(f)) for f in fields)
            u = fields[-1]
        return np.array(rows)

    def screen_points(self, u: np.ndarray, q: int, ms) -> np.ndarray:
        """The modal sum of screen q (times the absorber, before the
        reflection step) at the grid points ms only.  Same arithmetic as
        screen(): for each point only the rays that can land near it are
        marched, and the bracket found in that window is checked to have the
        whole stencil inside it (a landing order that would differ from the
        full ray family is an error, never silently used)."""
        g = self.g
        pb = self.pb
        u = self.project(u)
        c = self.modes(u)
        s_all = self.launch_points()
        kmax = g.n_max * (2.0 * math.pi / pb.k) / g.L
        reach = pb.dx * kmax / math.sqrt(1.0 - kmax * kmax)
        out = np.zeros(len(ms), dtype=np.complex128)
        for idx, m in enumerate(ms):
            zm = g.z_lo + g.dz * m
            half = int(math.ceil((2.0 * reach + 4 * g.R * g.dz) / (g.R * g.dz))) + 4
            while True:
                jc = int(np.searchsorted(s_all, zm))
                j0 = max(jc - half, 0)
                j1 = min(jc + half, g.NRT - 1)
                rays = self.march(q, self.kappa[:, None], s_all[None, j0:j1 + 1])
                delta = (rays["z"] - g.z_lo) / g.dz
                if np.any(np.diff(delta, axis=1) <= 0):
                    raise CausticError("ray landings not increasing (rays crossed)")
                jj = np.array([np.searchsorted(row, m, side="right") - 1 for row in delta])
                if jj.min() >= 1 and jj.max() <= delta.shape[1] - 3:
                    break
                if j0 == 0 and j1 == g.NRT - 1:
                    raise RangeError("ghost rays do not cover the screen")
                half *= 2
            acc = 0j
            for i in range(len(self.n)):
                j = jj[i]
                x = [delta[i, j + o] for o in (-1, 0, 1, 2)]
                vals = []
                for v in (rays["r"][i], rays["a"][i]):
                    f = [v[j + o] for o in (-1, 0, 1, 2)]
                    tot = 0.0
                    for p_ in range(4):
                        wgt = 1.0
                        for l_ in range(4):
                            if l_ != p_:
                                wgt *= (m - x[l_]) / (x[p_] - x[l_])
                        tot += wgt * f[p_]
                    vals.append(tot)
                n = int(self.n[i])
                base = 2.0 * math.pi * ((n * m) % g.N) / g.N
                acc += c[i] * vals[1] * np.exp(1j * (base + pb.k * vals[0]))
            out[idx] = acc * self.W[m]
        return out

    def propagate(self, u_phys: np.ndarray, q0: int = 0, n_screens: int | None = None,
                  snapshots: bool = False):
        """Screens q0 .. q0+n_screens-1 from the physical field on Gamma_{q0};
        returns the physical field on the last screen (and every screen's
        field when snapshots=True)."""
        if n_screens is None:
            n_screens = self.pb.n_screens
        u = self.extend(u_phys)
        snaps = []
        for q in range(q0, q0 + n_screens):
            u = self.screen(u, q)
            if snapshots:
                snaps.append(self.restrict(self.project(u)))
        res = self.restrict(self.project(u))
        return (res, snaps) if snapshots else res


def rel_l2(a, b) -> float:
    a = np.asarray(a)
    b = np.asarray(b)
    return float(np.linalg.norm(a - b) / max(np.linalg.norm(b), 1e-300))
