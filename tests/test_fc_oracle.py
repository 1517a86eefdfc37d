"""The Fourier-continuation oracle (Sec. 2.2) against its pins, then with
plausible mistakes planted (on the CPU, in altered copies) to show that each
is caught by at least one pin."""
import math

import numpy as np
import pytest

pytest.importorskip("mpmath")

import fc_pins as P  # noqa: E402
from oracle import fc_oracle as F  # noqa: E402
from oracle.swkb_oracle import Oracle, OracleError  # noqa: E402


@pytest.fixture(scope="module")
def tables():
    return F.fc_gram_tables()


# -- the oracle against its pins ------------------------------------------------

def test_gram_basis(tables):
    P.pin_gram_basis(tables[0])


def test_polynomials_reproduced(tables):
    P.pin_polynomials_reproduced(F.fc_extend, *tables)


def test_smooth_function_converges_at_high_order(tables):
    P.pin_smooth_convergence(F.fc_extend, *tables)


def test_periodic_function_reproduced(tables):
    P.pin_periodic_function(F.fc_extend, *tables)


def test_partition_of_unity():
    P.pin_partition(F.Patches, F.smooth_step)


def test_homogeneous_medium_against_angular_spectrum(tables):
    P.pin_homogeneous(F.FCOracle)


def test_homogeneous_closed_form(tables):
    P.pin_homogeneous_closed_form(F.FCOracle)


def test_planes_between_screens(tables):
    P.pin_planes_homogeneous(F.FCOracle)


def test_lens_against_periodic_swkb(tables):
    P.pin_against_periodic(F.FCOracle, Oracle)


def test_layout_and_cover_errors(tables):
    with pytest.raises(ValueError):
        F.Patches(300, 80, 16)                   # does not tile
    with pytest.raises(ValueError):
        F.Patches(272, 30, 16)                   # ramps would overlap
    pb = P.open_problem(144, 48, 3, 40.0, 0.0, 5.0)
    o = F.FCOracle(pb)
    assert o.patches.P == 3 and o.Np == 144 + 25
    assert o.n_max == math.floor(math.sin(pb.theta_max) * o.Np * P.STEP)
    # the march of a ray does not depend on the patch that launches it: the
    # same (kappa, z) gives the same landing from any patch's point of view
    s = o.launch_points()
    assert s[o.G] == pb.z_a and len(s) == pb.n_z + 2 * o.G


# -- planted mistakes ---------------------------------------------------------------

def extend_left_not_reversed(f, Q, A):
    d = Q.shape[0]
    f = np.asarray(f)
    right = A @ (Q.T @ f[len(f) - d:])
    left = A @ (Q.T @ f[:d])
    return np.concatenate([f, right + left])


def extend_project_with_Q(f, Q, A):
    d = Q.shape[0]
    f = np.asarray(f)
    right = A @ (Q @ f[len(f) - d:])
    left = A @ (Q @ f[d - 1::-1])
    return np.concatenate([f, right + left[::-1]])


def extend_right_only(f, Q, A):
    d = Q.shape[0]
    f = np.asarray(f)
    return np.concatenate([f, A @ (Q.T @ f[len(f) - d:])])


def _with_extend(ext):
    class V(F.FCOracle):
        def patch_modes(self, u):
            pt = self.patches
            out = np.empty((pt.P, len(self.n)), dtype=np.complex128)
            for p in range(pt.P):
                f = u[pt.start[p]:pt.start[p] + pt.n_pat]
                e = ext(f, self.Q, self.A)
                wv = np.fft.fft(e)
                out[p] = wv[self.n % len(e)] / len(e)
            return out
    return V


class PeriodFromPatchOnly(F.FCOracle):        # L_p = n_pat h: continuation left out of kappa
    def __init__(self, pb, tables=None):
        super().__init__(pb, tables)
        self.kappa = 2.0 * math.pi * self.n / (pb.k * pb.fc_patch * self.h)


class PhaseFromIntervalStart(F.FCOracle):    # every patch's series phased from z_a, not a_p
    def screen(self, u, q):
        pb = self.pb
        c = self.patch_modes(np.asarray(u, dtype=np.complex128))
        s = self.launch_points()
        rays = self.base.march(q, self.kappa[:, None], s[None, :])
        delta = (rays["z"] - pb.z_a) / self.h
        m = np.arange(pb.n_z)
        out = np.zeros(pb.n_z, dtype=np.complex128)
        for p in range(self.patches.P):
            S = self.patches.weight(p, (s - pb.z_a) / self.h)
            for i, n in enumerate(self.n):
                r_m, a_m = self.base.interpolate(delta[i], (rays["r"][i], S * rays["a"][i]))
                base = 2.0 * math.pi * ((int(n) * m) % self.Np) / self.Np
                out += c[p, i] * a_m * np.exp(1j * (base + pb.k * r_m))
        return out


class IndicatorWindow(F.FCOracle):           # S^p = 1 on the patch, 0 outside
    def __init__(self, pb, tables=None):
        super().__init__(pb, tables)
        pt = self.patches

        def indicator(p, u):
            u = np.asarray(u, dtype=np.float64)
            s = pt.start[p]
            lo = s if p > 0 else -np.inf
            hi = s + pt.n_pat - 1 if p < pt.P - 1 else np.inf
            # split the overlaps half and half so that the weights still sum to one
            if p > 0:
                lo = s + (pt.n_ov - 1) / 2.0
            if p < pt.P - 1:
                hi = s + pt.n_pat - 1 - (pt.n_ov - 1) / 2.0
            return ((u >= lo) & (u < hi)).astype(np.float64)
        pt.weight = indicator


class WindowAtTarget(F.FCOracle):            # S^p applied where the ray lands, not carried
    def screen(self, u, q):
        pb = self.pb
        c = self.patch_modes(np.asarray(u, dtype=np.complex128))
        s = self.launch_points()
        rays = self.base.march(q, self.kappa[:, None], s[None, :])
        delta = (rays["z"] - pb.z_a) / self.h
        m = np.arange(pb.n_z)
        out = np.zeros(pb.n_z, dtype=np.complex128)
        for p in range(self.patches.P):
            St = self.patches.weight(p, m.astype(np.float64))
            sp = int(self.patches.start[p])
            for i, n in enumerate(self.n):
                r_m, a_m = self.base.interpolate(delta[i], (rays["r"][i], rays["a"][i]))
                base = 2.0 * math.pi * ((int(n) * (m - sp)) % self.Np) / self.Np
                out += c[p, i] * St * a_m * np.exp(1j * (base + pb.k * r_m))
        return out


class ConjugateModes(F.FCOracle):            # w_{-n} taken for mode n
    def patch_modes(self, u):
        c = super().patch_modes(u)
        return c[:, ::-1]


def right_ramp_rises(Pt):
    class V(Pt):
        def weight(self, p, u):
            u = np.asarray(u, dtype=np.float64)
            s = self.start[p]
            e = s + self.n_pat - 1
            wdt = self.n_ov - 1
            return F.smooth_step((u - s) / wdt) * F.smooth_step((e - u) / wdt * 0.5)
    return V


def step_squared(t):                         # t^2 in place of the C-infinity step
    return np.clip(np.asarray(t, dtype=np.float64), 0.0, 1.0) ** 2


MUTANTS_TABLES = {
    "left-blend-not-reversed": extend_left_not_reversed,
    "gram-projection-with-Q": extend_project_with_Q,
    "left-end-not-continued": extend_right_only,
}


@pytest.mark.parametrize("name", sorted(MUTANTS_TABLES))
def test_continuation_mutants_are_caught(name, tables):
    ext = MUTANTS_TABLES[name]
    caught = []
    for pin in (P.pin_polynomials_reproduced, P.pin_smooth_convergence, P.pin_periodic_function):
        try:
            pin(ext, *tables)
        except AssertionError:
            caught.append(pin.__name__)
    assert caught, name


MUTANTS_ORACLE = {
    "period-without-continuation": PeriodFromPatchOnly,
    "phase-from-interval-start": PhaseFromIntervalStart,
    "indicator-window": IndicatorWindow,
    "window-at-target": WindowAtTarget,
    "conjugate-modes": ConjugateModes,
    "left-blend-not-reversed-in-screen": _with_extend(extend_left_not_reversed),
}


@pytest.mark.parametrize("name", sorted(MUTANTS_ORACLE))
def test_oracle_mutants_are_caught(name, tables):
    # a pin fails, or the mutant's rays become impossible (an evanescent mode)
    caught = []
    for pin in (P.pin_homogeneous, P.pin_homogeneous_closed_form):
        try:
            pin(MUTANTS_ORACLE[name])
        except (AssertionError, OracleError):
            caught.append(pin.__name__)
    assert caught, name


@pytest.mark.parametrize("name,pt,step", [
    ("right-ramp-rises", "right", F.smooth_step),
    ("step-squared", None, step_squared),
])
def test_partition_mutants_are_caught(name, pt, step):
    Pt = right_ramp_rises(F.Patches) if pt == "right" else F.Patches
    with pytest.raises(AssertionError):
        P.pin_partition(Pt, step)


def test_library_continuation_table_matches_the_oracle(tables):
    """The CUDA library builds its continuation operator with its own
    generator (Gram-Schmidt and normal equations in 100 digits); both are
    roundings of the same operator A Q^T (independent of the Gram
    polynomials' signs)."""
    import os
    import re
    path = os.path.join(os.path.dirname(__file__), "..", "paper_2301_03814_gb300", "csrc",
                        "swkb_fc_tables.h")
    txt = open(path).read()
    body = txt[txt.index("= {") + 3:txt.index("};")]
    lib = np.array([float(v) for v in re.findall(r"[-+]?\d\.\d+e[-+]\d+", body)])
    Q, A = tables
    want = A @ Q.T
    assert lib.shape == (want.size,)
    assert np.max(np.abs(lib.reshape(want.shape) - want)) <= 1e-15 * np.max(np.abs(want))


def test_screen_points_equal_the_whole_screen(tables):
    """The sampled form used at full size gives the whole screen's values:
    the same rays, brackets, weights and terms, summed in the same order."""
    pb = P.open_problem(144, 48, 3, 52.0, 6.0, 5.0, n_screens=1)
    o = F.FCOracle(pb)
    whole = o.screen(pb.u0, 0)
    ms = [0, 1, 47, 96, 120, 143, 190, 240, pb.n_z - 2, pb.n_z - 1]
    got = o.screen_points(pb.u0, 0, ms)
    assert np.max(np.abs(got - whole[ms])) <= 1e-13 * np.max(np.abs(whole))
