"""Plant plausible mistakes in the oracle (on the CPU, in subclasses) and
check that at least one pin catches each.  This is what makes the pins
evidence: a dropped term, a wrong sign or index, or a swapped operand
anywhere on the path must fail one of them."""
import math

import numpy as np
import pytest

import oracle_pins as P
from oracle.swkb_oracle import Oracle


class NoSqrtAmplitude(Oracle):            # paper's printed A = (J/J0) A0 form
    def march(self, q, kappa, s, steps=None):
        r = super().march(q, kappa, s, steps)
        r["a"] = r["a"] ** 2
        return r


class SwappedP0P1(Oracle):
    def march(self, q, kappa, s, steps=None):
        r = super().march(q, kappa, s, steps)
        r["a"] = np.sqrt(r["P1"] / (r["P0"] * r["Zs"]))
        return r


class PlanesMarchWholeScreen(Oracle):     # planes reuse the screen's landing
    def march(self, q, kappa, s, steps=None):
        return super().march(q, kappa, s)


class PlanesWithAbsorber(Oracle):         # absorber applied between screens too
    def screen_planes(self, u, q, planes):
        return [f * self.W for f in super().screen_planes(u, q, planes)[:-1]] + \
            super().screen_planes(u, q, planes)[-1:]


def _rhs_variant(kind):
    class V(Oracle):
        def rhs(self, xs, kappa, z, Q, r, Zs, Qs):
            x, right = xs
            e, ez, ezz = self.medium.eval(x, right, z)
            P = np.sqrt(e - Q * Q)
            dz = Q / P
            dQ = ez / (2.0 * P) if kind != "dQ-factor" else ez / P
            dr = (e - kappa * Q) / P if kind != "dr-kappa2" else (e - kappa * kappa) / P
            Ps = (ez * Zs - 2.0 * Q * Qs) / (2.0 * P) if kind != "Ps-sign" else (ez * Zs + 2.0 * Q * Qs) / (2.0 * P)
            dZs = (Qs - Q * Ps / P) / P
            dQs = ezz * Zs / (2.0 * P) - (ez * Ps / (2.0 * P * P) if kind != "Qs-drop" else 0.0)
            return dz, dQ, dr, dZs, dQs
    return V


class SwappedBlendWeight(Oracle):        # th <-> 1 - th between range columns
    def __init__(self, pb):
        super().__init__(pb)
        base = self.medium.column_weights

        def swapped(x, right):
            c, th = base(x, right)
            return c, 1.0 - th
        self.medium.column_weights = swapped


class SwappedColumnLimits(Oracle):        # left limit at a screen start, right at its end
    def __init__(self, pb):
        super().__init__(pb)
        base = self.medium.column_weights
        self.medium.column_weights = lambda x, right: base(x, not right)


class BlendWeightOnlyInside(Oracle):      # the blend formula itself with swapped weights
    def __init__(self, pb):
        super().__init__(pb)
        m = self.medium
        plain = m.eval

        def ev(x, right, z):
            c, th = m.column_weights(x, right)
            if th in (0.0, 1.0):
                return plain(x, right, z)
            a = m.column_eval(c, z)
            b = m.column_eval(c + 1, z)
            return tuple(th * a[i] + (1.0 - th) * b[i] for i in range(3))
        m.eval = ev


class ConjugateDFT(Oracle):
    def modes(self, u):
        return np.fft.ifft(u)[self.n % self.g.N]


class ShiftedOrigin(Oracle):              # psi_n origin one grid cell off
    def modes(self, u):
        return super().modes(u) * np.exp(2j * math.pi * self.n / self.g.N)


class ShiftedStencil(Oracle):              # stencil j..j+3 instead of j-1..j+2
    def interpolate(self, delta, vals):
        m = np.arange(self.g.N, dtype=np.float64)
        j = np.searchsorted(delta, m, side="right") - 1
        x = [delta[j + o] for o in (0, 1, 2, 3)]
        out = []
        for v in vals:
            f = [v[j + o] for o in (0, 1, 2, 3)]
            acc = np.zeros(self.g.N)
            for p in range(4):
                wgt = np.ones(self.g.N)
                for l in range(4):
                    if l != p:
                        wgt = wgt * (m - x[l]) / (x[p] - x[l])
                acc = acc + wgt * f[p]
            out.append(acc)
        return out


def _caught(O):
    checks = [
        lambda: P.pin_modes_bruteforce(O) > 1e-13,
        lambda: P.pin_homogeneous(O, eps0=1.1, R=2) > 1e-12,
        lambda: P.pin_homogeneous(O, bc=1) > 1e-12,
        lambda: P.pin_linear_ray(O, 64) > 1e-9,
        lambda: P.pin_tube_flux(O) > 1e-6,
        lambda: P.pin_tube_flux(O, x_dependent=True) > 1e-6,
        lambda: P.pin_interp_stencil(O) > 1e-9,
        lambda: P.pin_planes_homogeneous(O) > 1e-12,
        lambda: P.pin_planes_homogeneous(O, bc=1) > 1e-12,
        lambda: P.pin_linear_ray_steps(O) > 1e-7,
        lambda: P.pin_planes_before_absorber(O) > 1e-12,
        lambda: P.pin_x_only_columns(O) > 1e-9,
    ]
    for c in checks:
        try:
            if c():
                return True
        except Exception:
            return True
    return False


@pytest.mark.parametrize("O", [NoSqrtAmplitude, SwappedP0P1, _rhs_variant("dQ-factor"),
                               _rhs_variant("dr-kappa2"), _rhs_variant("Ps-sign"),
                               _rhs_variant("Qs-drop"), ConjugateDFT, ShiftedOrigin,
                               ShiftedStencil, PlanesMarchWholeScreen, PlanesWithAbsorber,
                               SwappedBlendWeight, SwappedColumnLimits, BlendWeightOnlyInside],
                         ids=["amp-no-sqrt", "P0-P1-swap", "dQ-factor", "dr-kappa2", "Ps-sign",
                              "Qs-drop", "conj-dft", "origin-shift", "stencil-shift",
                              "planes-whole-screen", "planes-absorbed", "blend-swapped",
                              "limits-swapped", "blend-formula-swapped"])
def test_planted_mistake_is_caught(O):
    assert _caught(O)


def test_unmutated_oracle_passes_all_checks():
    assert not _caught(Oracle)
