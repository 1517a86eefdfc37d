"""Plain, slow FP64 CPU oracle of the overlapping Fourier-continuation S-WKB.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU-baseline leg
of the benchmark may import this module.  The CUDA library never calls it and
shares no code with it (it builds its own continuation tables).

What it computes (Bruno & Maas, Sec. 2.2, Eq. ifft_eq_phi_patches): on a
non-periodic interval [z_a, z_b) whose field vanishes near both ends, the
screen field is split into overlapping patches; on each patch a Fourier
continuation (FC) gives a Fourier series of the field's restriction, a smooth
partition of unity S^p that vanishes at the patch ends weights the patches,
and every mode of every patch is carried across the screen by the rays of the
periodic method (Sec. 2.1.2) with launch amplitude S^p(z) w_n^p / N.

Readings (the section gives a sketch; where it is silent this is the choice):

  F1  patches: the physical grid z_m = z_a + m h, m = 0..n_z-1, h =
      (z_b - z_a) / n_z.  Patch p holds the n_pat grid points s_p .. e_p,
      s_p = p (n_pat - n_ov), e_p = s_p + n_pat - 1; neighbours share n_ov
      points; the patches tile the grid exactly, n_z = s_{P-1} + n_pat, and
      n_pat >= 2 n_ov.
  F2  partition of unity: with the C-infinity step r(t) = e^{-1/t} /
      (e^{-1/t} + e^{-1/(1-t)}) (0 for t <= 0, 1 for t >= 1) and u the
      position in grid units, S^p(u) = r((u - s_p) / (n_ov - 1))
      (1 - r((u - e_p + n_ov - 1) / (n_ov - 1))).  On an overlap the two
      patches' weights are r and 1 - r of the same t, so they sum to one;
      every S^p vanishes at both ends of its patch and outside it; the sum is
      below one only on the first and last n_ov - 1 points of the interval,
      where the field must vanish.
  F3  continuation: FC-Gram (Bruno & Lyon 2010; Albin & Bruno 2011).  The d
      end values of a patch at each end are expanded in the Gram polynomials
      orthonormal on d equispaced points; each Gram polynomial has a
      precomputed blend-to-zero continuation over C points: the trigonometric
      polynomial of period 2 (d + C) grid steps with H harmonics fitting, by
      least squares on points oversampled o times per step, the polynomial on
      [0, d - 1] and zero on [d + C, 2 d + C - 1], evaluated at d .. d + C - 1.
      d = 5, C = 25, H = 12, o = 20, fitted in 60-digit arithmetic and rounded
      to FP64.  The patch's N_p = n_pat + C point periodic sequence is the
      samples followed by the right end's blend plus the mirrored blend of
      the left end.
  F4  modes: w_n^p = DFT of that sequence (Eq. fft_eq with N = N_p), the
      series (1/N_p) sum_n w_n^p exp(2 pi i n (z - a_p) / L_p), a_p = z_a +
      s_p h, L_p = N_p h, kappa_n = 2 pi n / (k L_p); kept |n| <= n_max =
      min(floor(sin(theta_max) L_p / lambda), N_p / 2 - 1) (n_max > 0 in the
      problem overrides), as in the periodic method.  All patches have the
      same N_p and so the same kappa_n.
  F5  rays: every patch launches its rays from the interval's one launch
      grid z_j = z_a + (j - G) R h, j = 0 .. n_z / R + 2 G - 1, with
      G = ceil(dx tan(theta_top) / (R h)) + 3 ghost rays beyond each end
      (theta_top the steepest kept mode's angle); ray (n, j) of patch p
      starts with amplitude S^p(z_j) w_n^p / N_p (zero outside the patch) and
      phase k kappa_n (z_j - a_p).  A ray's march (Eqs. charsys, charsys_s,
      transport_xt, the periodic readings R5-R7, R10) depends only on
      (kappa_n, z_j), so one march per (mode, launch point) serves every
      patch.  The medium table must cover the ghosts and the landings.
  F6  resummation: per patch and mode, the residual phase r and the
      amplitude S^p(z_j) sqrt(P0 / (P1 Z_s)) are interpolated from the
      landings onto the n_z grid points exactly as in the periodic method
      (R8: bracket delta_j <= m < delta_{j+1}, 4-point Lagrange), and
      u(z_m) = sum_p sum_n (w_n^p / N_p) A exp(i (2 pi n (m - s_p) / N_p + k r)).
      Grid points outside the ghosts' cover are an error.  Fields between
      screens follow the periodic reading R15: the screen's patch modes,
      their rays stopped on the plane, the same sum.

Everything is float64 except the continuation tables, which are computed in
extended precision (mpmath) and then rounded.
"""
from __future__ import annotations

import functools
import math

import numpy as np

from .swkb_oracle import PERIODIC, CausticError, Oracle, RangeError

OPEN = 3

FC_D = 5            # matching points at each patch end
FC_C = 25           # continuation points
FC_HARMONICS = 12   # harmonics of the blend-to-zero fit
FC_OVERSAMPLE = 20  # fitting points per grid step
FC_DIGITS = 60      # working precision of the table construction


# ----------------------------------------------------------------------------
# F3: FC-Gram continuation tables
# ----------------------------------------------------------------------------

@functools.lru_cache(maxsize=None)
def fc_gram_tables(d: int = FC_D, C: int = FC_C, harmonics: int = FC_HARMONICS,
                   oversample: int = FC_OVERSAMPLE, digits: int = FC_DIGITS):
    """(Q, A): Q (d x d), column j the values at x = 0 .. d-1 of the Gram
    polynomial q_j (orthonormal in the discrete inner product on these points:
    Gram-Schmidt of 1, x, .., x^{d-1}, i.e. the QR factorisation of the
    Vandermonde matrix V = Q R, so q_j(x) = sum_k x^k (R^-1)_{kj}); A (C x d),
    column j the blend-to-zero continuation of q_j at x = d .. d+C-1 (F3)."""
    import mpmath as mp

    with mp.workdps(digits):
        V = mp.matrix(d, d)
        for i in range(d):
            for k in range(d):
                V[i, k] = mp.mpf(i) ** k
        Q, R = mp.qr(V)
        Rinv = R ** -1
        period = 2 * (d + C)
        match = [mp.mpf(i) / oversample for i in range((d - 1) * oversample + 1)]
        zero = [mp.mpf(d + C) + mp.mpf(i) / oversample for i in range((d - 1) * oversample + 1)]
        pts = match + zero

        def basis_row(x):
            row = [mp.mpf(1)]
            for m in range(1, harmonics + 1):
                th = 2 * mp.pi * m * x / period
                row += [mp.cos(th), mp.sin(th)]
            return row

        F = mp.matrix([basis_row(x) for x in pts])
        Ad = np.empty((C, d))
        for j in range(d):
            rhs = mp.matrix(len(pts), 1)
            for r, x in enumerate(match):
                rhs[r] = mp.fsum(Rinv[k, j] * x ** k for k in range(d))
            coef, _ = mp.qr_solve(F, rhs)
            for i in range(C):
                row = basis_row(mp.mpf(d + i))
                Ad[i, j] = float(mp.fsum(row[c] * coef[c] for c in range(len(row))))
        Qd = np.array([[float(Q[i, j]) for j in range(d)] for i in range(d)])
    return Qd, Ad


def fc_extend(f: np.ndarray, Q: np.ndarray, A: np.ndarray) -> np.ndarray:
    """The N_p = n + C point periodic sequence of F3 for samples f[0..n-1]:
    f, then the continuation past f[n-1] (right end's Gram coefficients
    Q^T f[n-d..n-1] through A) plus the continuation before f[0] (the left
    end read backwards, f[d-1], .., f[0], through A, placed in reverse)."""
    d = Q.shape[0]
    f = np.asarray(f)
    right = A @ (Q.T @ f[len(f) - d:])
    left = A @ (Q.T @ f[d - 1::-1])
    return np.concatenate([f, right + left[::-1]])


# ----------------------------------------------------------------------------
# F1 / F2: patches and the partition of unity
# ----------------------------------------------------------------------------

def smooth_step(t):
    """r(t) = e^{-1/t} / (e^{-1/t} + e^{-1/(1-t)}), 0 for t <= 0, 1 for t >= 1."""
    t = np.asarray(t, dtype=np.float64)
    out = np.where(t >= 1.0, 1.0, 0.0)
    inner = (t > 0.0) & (t < 1.0)
    ti = t[inner]
    a = np.exp(-1.0 / ti)
    b = np.exp(-1.0 / (1.0 - ti))
    out[inner] = a / (a + b)
    return out


class Patches:
    """F1 layout and F2 weights for n_z grid points."""

    def __init__(self, n_z: int, n_pat: int, n_ov: int):
        if n_ov < 2 or n_pat < 2 * n_ov or n_pat > n_z:
            raise ValueError("need 2 <= n_ov, 2 n_ov <= n_pat <= n_z")
        stride = n_pat - n_ov
        if (n_z - n_pat) % stride:
            raise ValueError("patches must tile the grid: (n_z - n_pat) % (n_pat - n_ov) == 0")
        self.n_z, self.n_pat, self.n_ov = n_z, n_pat, n_ov
        self.P = (n_z - n_pat) // stride + 1
        self.start = np.arange(self.P) * stride

    def weight(self, p: int, u) -> np.ndarray:
        """S^p at grid-unit positions u."""
        u = np.asarray(u, dtype=np.float64)
        s = self.start[p]
        e = s + self.n_pat - 1
        w = self.n_ov - 1
        return smooth_step((u - s) / w) * (1.0 - smooth_step((u - (e - w)) / w))


# ----------------------------------------------------------------------------
# the propagator
# ----------------------------------------------------------------------------

class FCOracle:
    def __init__(self, pb, tables=None):
        if pb.bc != OPEN:
            raise ValueError("the continuation path is for non-periodic (open) intervals")
        self.pb = pb
        self.h = (pb.z_b - pb.z_a) / pb.n_z
        self.patches = Patches(pb.n_z, pb.fc_patch, pb.fc_overlap)
        self.Q, self.A = fc_gram_tables() if tables is None else tables
        self.C = self.A.shape[0]
        self.Np = pb.fc_patch + self.C
        self.Lp = self.Np * self.h
        lam = 2.0 * math.pi / pb.k
        if pb.n_max > 0:
            n_max = int(pb.n_max)
        else:
            n_max = int(math.floor(math.sin(pb.theta_max) * self.Lp / lam * (1.0 + 1e-12)))
        self.n_max = min(n_max, self.Np // 2 - 1)
        self.n = np.arange(-self.n_max, self.n_max + 1)
        self.kappa = 2.0 * math.pi * self.n / (pb.k * self.Lp)
        R = int(pb.ray_stride)
        if pb.n_z % R:
            raise ValueError("ray stride must divide n_z")
        self.R = R
        kmax = self.n_max * lam / self.Lp
        tan_t = kmax / math.sqrt(1.0 - kmax * kmax)
        self.G = int(math.ceil(pb.dx * tan_t / (R * self.h) - 1e-9)) + 3
        self.NRT = pb.n_z // R + 2 * self.G
        # the periodic oracle on the same grid supplies the medium, the RK4
        # march and the Lagrange interpolation (its own mode set is unused)
        self.base = Oracle(pb.with_(bc=PERIODIC, n_max=1))

    def launch_points(self) -> np.ndarray:
        j = np.arange(self.NRT)
        return self.pb.z_a + (j - self.G) * self.R * self.h

    def patch_modes(self, u: np.ndarray) -> np.ndarray:
        """[P][2 n_max + 1]: w_n^p / N_p of every patch (F3, F4)."""
        pt = self.patches
        out = np.empty((pt.P, len(self.n)), dtype=np.complex128)
        for p in range(pt.P):
            f = u[pt.start[p]:pt.start[p] + pt.n_pat]
            w = np.fft.fft(fc_extend(f, self.Q, self.A))
            out[p] = w[self.n % self.Np] / self.Np
        return out

    def screen(self, u: np.ndarray, q: int) -> np.ndarray:
        """Gamma_q -> Gamma_{q+1} on the n_z grid points (F1-F6)."""
        u = np.asarray(u, dtype=np.complex128)
        return self.ray_sum(self.patch_modes(u), q, None)

    def screen_planes(self, u: np.ndarray, q: int, planes: int):
        """Fields of screen q on the planes x_q + j dx / planes, j = 1..planes
        (the periodic oracle's R15 applied to the patches): the screen's
        patch modes, their rays marched j rk4_steps / planes steps, summed as
        on the screen.  The last plane is the screen's own field."""
        pb = self.pb
        if planes < 1 or pb.rk4_steps % planes:
            raise ValueError("planes must divide rk4_steps")
        c = self.patch_modes(np.asarray(u, dtype=np.complex128))
        return [self.ray_sum(c, q, j * pb.rk4_steps // planes) for j in range(1, planes + 1)]

    def propagate_planes(self, u0: np.ndarray, q0: int, n_screens: int, planes: int):
        """Fields on every plane of screens q0 .. q0+n_screens-1, rows ordered
        (screen, plane); each screen starts from the previous screen's last
        plane."""
        u = np.asarray(u0, dtype=np.complex128)
        rows = []
        for q in range(q0, q0 + n_screens):
            fields = self.screen_planes(u, q, planes)
            rows.extend(fields)
            u = fields[-1]
        return np.array(rows)

    def ray_sum(self, c: np.ndarray, q: int, steps) -> np.ndarray:
        """Eq. ifft_eq_phi_patches carried to the plane reached after `steps`
        RK4 steps of screen q (None: the next screen), F5-F6."""
        pb = self.pb
        s = self.launch_points()
        rays = self.base.march(q, self.kappa[:, None], s[None, :], steps=steps)
        delta = (rays["z"] - pb.z_a) / self.h
        u_launch = (s - pb.z_a) / self.h
        m = np.arange(pb.n_z)
        out = np.zeros(pb.n_z, dtype=np.complex128)
        for p in range(self.patches.P):
            S = self.patches.weight(p, u_launch)
            sp = int(self.patches.start[p])
            for i, n in enumerate(self.n):
                r_m, a_m = self.base.interpolate(delta[i], (rays["r"][i], S * rays["a"][i]))
                base = 2.0 * math.pi * ((int(n) * (m - sp)) % self.Np) / self.Np
                out += c[p, i] * a_m * np.exp(1j * (base + pb.k * r_m))
        return out

    def screen_points(self, u: np.ndarray, q: int, ms) -> np.ndarray:
        """screen() at the grid points ms only, for fields too large for the
        whole screen: the same patch modes, and for each point only the rays
        launched near it (a window of the launch grid that the steepest kept
        mode cannot cross in one screen, widened until every mode's stencil
        around the point lies inside it); per patch and mode the same bracket,
        Lagrange weights and term as screen(), added in the same order."""
        pb = self.pb
        u = np.asarray(u, dtype=np.complex128)
        c = self.patch_modes(u)
        s_all = self.launch_points()
        lam = 2.0 * math.pi / pb.k
        kmax = self.n_max * lam / self.Lp
        reach = pb.dx * kmax / math.sqrt(1.0 - kmax * kmax)
        out = np.zeros(len(ms), dtype=np.complex128)
        for idx, m in enumerate(ms):
            half = int(math.ceil((reach + 4 * self.R * self.h) / (self.R * self.h))) + 4
            while True:
                jc = int(np.searchsorted(s_all, pb.z_a + self.h * m))
                j0 = max(jc - half, 0)
                j1 = min(jc + half, self.NRT - 1)
                s = s_all[j0:j1 + 1]
                rays = self.base.march(q, self.kappa[:, None], s[None, :])
                delta = (rays["z"] - pb.z_a) / self.h
                if np.any(np.diff(delta, axis=1) <= 0):
                    raise CausticError("ray landings not increasing (rays crossed)")
                jj = np.array([np.searchsorted(row, m, side="right") - 1 for row in delta])
                if jj.min() >= 1 and jj.max() <= delta.shape[1] - 3:
                    break
                if j0 == 0 and j1 == self.NRT - 1:
                    raise RangeError("ghost rays do not cover the screen")
                half *= 2
            u_launch = (s - pb.z_a) / self.h
            acc = 0j
            for p in range(self.patches.P):
                S = self.patches.weight(p, u_launch)
                if not np.any(S):
                    continue            # every term of this patch is exactly zero here
                sp = int(self.patches.start[p])
                for i, n in enumerate(self.n):
                    j = jj[i]
                    x = [delta[i, j + o] for o in (-1, 0, 1, 2)]
                    vals = []
                    for v in (rays["r"][i], S * rays["a"][i]):
                        f = [v[j + o] for o in (-1, 0, 1, 2)]
                        tot = 0.0
                        for a in range(4):
                            wgt = 1.0
                            for b in range(4):
                                if b != a:
                                    wgt *= (m - x[b]) / (x[a] - x[b])
                            tot += wgt * f[a]
                        vals.append(tot)
                    base = 2.0 * math.pi * ((int(n) * (m - sp)) % self.Np) / self.Np
                    acc += c[p, i] * vals[1] * np.exp(1j * (base + pb.k * vals[0]))
            out[idx] = acc
        return out

    def propagate(self, u0: np.ndarray, q0: int = 0, n_screens: int | None = None,
                  snapshots: bool = False):
        if n_screens is None:
            n_screens = self.pb.n_screens
        u = np.asarray(u0, dtype=np.complex128)
        snaps = []
        for q in range(q0, q0 + n_screens):
            u = self.screen(u, q)
            if snapshots:
                snaps.append(u.copy())
        return (u, snaps) if snapshots else u


__all__ = ["FCOracle", "Patches", "fc_gram_tables", "fc_extend", "smooth_step", "OPEN",
           "RangeError"]
