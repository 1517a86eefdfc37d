"""Pins of the separation-of-variables oracle (oracle/hill_oracle.py), no GPU.

The references are independent of the oracle's construction: Mathieu
characteristic values and functions (scipy.special, the exact eigenpairs
for eps = eps0 + eps1 cos(2 kappa_1 s)), the angular spectrum for a
homogeneous medium, unitarity, and the full complex Fourier (Hill) matrix
of refs.hill_one_way on the whole period, which needs neither the parity
split nor the cosine/sine weights.  A planted mistake in any step of the
oracle fails one of them (the mutation tests at the end)."""
import contextlib
import math

import numpy as np
import pytest
import scipy.special as sp

from oracle import hill_oracle as H
from oracle.swkb_oracle import rel_l2
from paper_2301_03814_gb300 import workloads as w
from refs import angular_spectrum, hill_one_way


def _mathieu_case():
    """k = 2 pi, period 8 (H = 4 over a Neumann / Dirichlet ground),
    eps = 1 - 0.05 cos(4 pi s / L): Mathieu's equation with q = 1.6."""
    k, Hh, eps0, eps1 = 2.0 * math.pi, 4.0, 1.0, -0.05
    L = 2.0 * Hh
    q = -(L / (2.0 * math.pi)) ** 2 * k * k * eps1 / 2.0
    n_q = 512
    s = np.arange(n_q + 1) * Hh / n_q
    return k, Hh, L, eps0, q, eps0 + eps1 * np.cos(4.0 * math.pi * s / L)


def pin_mathieu_eigenvalues(mod=H):
    k, Hh, L, eps0, q, eps = _mathieu_case()
    K = 40
    eh = mod.cosine_coefficients(eps, 2 * K + 1)
    err = 0.0
    for par, f, ms in (("even", sp.mathieu_a, range(0, 10)), ("odd", sp.mathieu_b, range(1, 10))):
        A, _, _ = mod.hill_matrix(k, L, eh, K, par)
        lam = np.sort(np.linalg.eigvalsh(A))[::-1]
        want = np.array([k * k * eps0 - (2.0 * math.pi / L) ** 2 * f(m, q) for m in ms])
        err = max(err, np.max(np.abs(lam[:len(want)] - want)) / np.max(np.abs(want)))
    return err


def pin_mathieu_mode_phase(mod=H, bc=H.BC_PERIODIC, m=2, odd=False, x=37.0):
    """A Mathieu function as the field: it only gains exp(i alpha x).  The
    periodic layout samples the whole period [-H, H) about z_c = 0 (cosines
    and sines both); the Dirichlet layout samples [0, H) and mirrors it oddly
    (se_m vanishes at the top point, which the grounded period sets to 0)."""
    k, Hh, L, eps0, q, eps = _mathieu_case()
    if bc == H.BC_PERIODIC:
        n_z, z_a = 512, -Hh
    else:
        n_z, z_a, odd = 256, 0.0, True
    z = z_a + np.arange(n_z) * (2.0 * Hh if bc == H.BC_PERIODIC else Hh) / n_z
    deg = np.degrees(2.0 * math.pi * z / L)
    if odd:
        u0 = sp.mathieu_sem(m, q, deg)[0].astype(complex)
        a = sp.mathieu_b(m, q)
    else:
        u0 = sp.mathieu_cem(m, q, deg)[0].astype(complex)
        a = sp.mathieu_a(m, q)
    alpha = math.sqrt(k * k * eps0 - (2.0 * math.pi / L) ** 2 * a)
    got = mod.propagate(k, eps, u0, [x], bc, z_a, Hh, 40, z_c=0.0)[0]
    return rel_l2(got, np.exp(1j * alpha * x) * u0)


def pin_homogeneous(mod=H, bc=H.BC_NEUMANN):
    """eps = 1.05 everywhere: the angular spectrum of the mirrored field."""
    k, Hh, n_z, K, x = 2.0 * math.pi, 32.0, 256, 40, 23.0
    rng = np.random.default_rng(7)
    z = np.arange(n_z) * Hh / n_z
    u0 = np.exp(-((z - 9.0) / 2.5) ** 2) * np.exp(1j * rng.uniform(0, 2 * math.pi))
    if bc == H.BC_DIRICHLET:
        u0 = u0 * np.sin(math.pi * z / Hh)
    got = mod.propagate(k, np.full(2 * K + 1, 1.05), u0, [x], bc, 0.0, Hh, K)[0]
    full = H.field_on_period(u0, bc, n_z)
    want = angular_spectrum(full, k, 2.0 * Hh, x, K, eps0=1.05)[n_z:]
    return rel_l2(got, want)


def _duct(n_z=1024, height=25.0):
    pb = w.config_surface_duct_small(n_z=n_z, height=height)
    f = w.f_trilinear_duct(pb.meta["z_t"], pb.meta["g_d"])
    return pb, lambda z: f(np.asarray(z))[0]


def pin_full_fourier(mod=H, bc=H.BC_NEUMANN, x=300.0):
    """The parity-split problem against the full complex Hill matrix of the
    whole period (refs.hill_one_way) on the same eps samples."""
    pb, eps = _duct()
    Hh, n_z, K = pb.z_b - pb.z_a, pb.n_z, 160
    n_q = 2 * K
    s = np.arange(n_q + 1) * Hh / n_q
    u0 = pb.u0 if bc == H.BC_NEUMANN else pb.u0 * np.sin(math.pi * np.arange(n_z) / n_z)
    got = mod.propagate(pb.k, eps(s), u0, [x], bc, pb.z_a, pb.z_b, K)[0]
    full = H.field_on_period(u0, bc, n_z)
    ref = hill_one_way(full, pb.k, 2.0 * Hh, lambda t: eps(np.abs(t - Hh)), x, K,
                       n_quad=2 * n_q)[n_z:]
    return rel_l2(got, ref)


def pin_full_fourier_periodic(mod=H, x=40.0):
    """A Gaussian layer even about the middle of a periodic domain."""
    k, L, n_z, K = 2.0 * math.pi, 64.0, 512, 100
    n_q = 2 * K
    f = lambda t: 1.0 + 0.02 * np.exp(-0.01 * (t - L / 2) ** 2)
    s = L / 2 + np.arange(n_q + 1) * L / (2 * n_q)
    z = np.arange(n_z) * L / n_z
    u0 = np.exp(-((z - 20.0) / 3.0) ** 2) * np.exp(1j * 0.3 * k * z)
    got = mod.propagate(k, f(s), u0, [x], H.BC_PERIODIC, 0.0, L, K, z_c=L / 2)[0]
    ref = hill_one_way(u0, k, L, f, x, K, n_quad=2 * n_q)
    return rel_l2(got, ref)


def pin_unitary(mod=H, x=500.0):
    """No evanescent mode (K below the cut-off n = k L sqrt(eps_min) / 2 pi
    = 64): over the whole period (the periodic layout returns every point)
    the field keeps the norm of its band-limited part at x = 0."""
    k, L, n_z, K = 2.0 * math.pi, 64.0, 512, 50
    f = lambda t: 1.0 + 0.02 * np.exp(-0.01 * (t - L / 2) ** 2)
    s = L / 2 + np.arange(2 * K + 1) * L / (4 * K)
    z = np.arange(n_z) * L / n_z
    u0 = np.exp(-((z - 20.0) / 3.0) ** 2) * np.exp(1j * 0.3 * k * z)
    u = mod.propagate(k, f(s), u0, [0.0, x], H.BC_PERIODIC, 0.0, L, K, z_c=L / 2)
    return abs(np.linalg.norm(u[1]) / np.linalg.norm(u[0]) - 1.0)


def test_mathieu_eigenvalues():
    assert pin_mathieu_eigenvalues() < 1e-12


@pytest.mark.parametrize("bc,m,odd", [(H.BC_PERIODIC, 0, False), (H.BC_PERIODIC, 3, False),
                                      (H.BC_PERIODIC, 1, True), (H.BC_PERIODIC, 4, True),
                                      (H.BC_DIRICHLET, 1, True), (H.BC_DIRICHLET, 4, True)])
def test_mathieu_function_gains_its_phase(bc, m, odd):
    assert pin_mathieu_mode_phase(bc=bc, m=m, odd=odd) < 1e-9


@pytest.mark.parametrize("bc", [H.BC_NEUMANN, H.BC_DIRICHLET])
def test_homogeneous_is_the_angular_spectrum(bc):
    assert pin_homogeneous(bc=bc) < 1e-12


@pytest.mark.parametrize("bc", [H.BC_NEUMANN, H.BC_DIRICHLET])
def test_matches_the_full_fourier_hill_matrix(bc):
    assert pin_full_fourier(bc=bc) < 1e-10


def test_periodic_symmetric_matches_the_full_fourier_hill_matrix():
    assert pin_full_fourier_periodic() < 1e-10


def test_unitary_without_evanescent_modes():
    assert pin_unitary() < 1e-12


def test_x_zero_is_the_band_limited_field():
    pb, eps = _duct(n_z=256, height=4.0)
    K = 100
    s = np.arange(2 * K + 1) * (pb.z_b - pb.z_a) / (2 * K)
    u = H.propagate(pb.k, eps(s), pb.u0, [0.0], H.BC_NEUMANN, pb.z_a, pb.z_b, K)[0]
    full = H.field_on_period(pb.u0, H.BC_NEUMANN, pb.n_z)
    n = np.rint(np.fft.fftfreq(len(full), 1.0 / len(full)))
    want = np.fft.ifft(np.where(np.abs(n) <= K, np.fft.fft(full), 0.0))[pb.n_z:]
    assert rel_l2(u, want) < 1e-12


def test_rejects_bad_arguments():
    with pytest.raises(ValueError):
        H.propagate(1.0, np.ones(5), np.ones(16, complex), [1.0], H.BC_NEUMANN, 0.0, 1.0, 4)
    with pytest.raises(ValueError):
        H.propagate(1.0, np.ones(9), np.ones(16, complex), [1.0], H.BC_PERIODIC, 0.0, 1.0, 4,
                    z_c=0.03)


# --------------------------------------------------------------------------
# planted mistakes: each variant of the oracle must fail at least one pin
# --------------------------------------------------------------------------
ORIG = {name: getattr(H, name) for name in
        ("cosine_coefficients", "hill_matrix", "field_on_period", "basis")}


@contextlib.contextmanager
def planted(**override):
    """The oracle module with functions replaced for the duration."""
    for name, fn in override.items():
        setattr(H, name, fn)
    try:
        yield H
    finally:
        for name in override:
            setattr(H, name, ORIG[name])


def _hill_plus_for_sines(k, L, eh, K, parity):
    A, n, wt = ORIG["hill_matrix"](k, L, eh, K, "even")
    if parity == "odd":
        A, n, wt = A[1:, 1:], n[1:], wt[1:]
    return A, n, wt


def _hill_no_weights(k, L, eh, K, parity):
    A, n, wt = ORIG["hill_matrix"](k, L, eh, K, parity)
    if parity == "even":
        A = A.copy()
        A[0, 1:] /= math.sqrt(2.0)
        A[1:, 0] /= math.sqrt(2.0)
    return A, n, wt


def _hill_wrong_kappa(k, L, eh, K, parity):
    return ORIG["hill_matrix"](k, 2.0 * L, eh, K, parity)


def _coef_no_endpoint(eps_half, n_out):
    e = np.array(eps_half, float)
    e[-1] = e[-2]
    return ORIG["cosine_coefficients"](e, n_out)


def _mirror_sign_lost(u, bc, n_z):
    return ORIG["field_on_period"](u, H.BC_NEUMANN if bc == H.BC_DIRICHLET else bc, n_z)


def _basis_shifted(parity, n, w_, N, m_c):
    return ORIG["basis"](parity, n, w_, N, m_c + 1)


MUTANTS = {
    "sines use the cosine sum": dict(hill_matrix=_hill_plus_for_sines),
    "no sqrt(2) on the constant mode": dict(hill_matrix=_hill_no_weights),
    "kappa on twice the period": dict(hill_matrix=_hill_wrong_kappa),
    "last eps sample dropped": dict(cosine_coefficients=_coef_no_endpoint),
    "Dirichlet mirrored evenly": dict(field_on_period=_mirror_sign_lost),
    "basis off by one point": dict(basis=_basis_shifted),
}


def _pins_fail(mod):
    checks = [
        lambda: pin_mathieu_eigenvalues(mod) > 1e-9,
        lambda: pin_mathieu_mode_phase(mod, H.BC_PERIODIC, 2) > 1e-6,
        lambda: pin_mathieu_mode_phase(mod, H.BC_PERIODIC, 3, odd=True) > 1e-6,
        lambda: pin_mathieu_mode_phase(mod, H.BC_DIRICHLET, 3) > 1e-6,
        lambda: pin_homogeneous(mod, H.BC_NEUMANN) > 1e-9,
        lambda: pin_homogeneous(mod, H.BC_DIRICHLET) > 1e-9,
        lambda: pin_full_fourier(mod, H.BC_NEUMANN) > 1e-7,
        lambda: pin_full_fourier(mod, H.BC_DIRICHLET) > 1e-7,
        lambda: pin_full_fourier_periodic(mod) > 1e-7,
    ]
    return [c() for c in checks]


@pytest.mark.parametrize("name", sorted(MUTANTS))
def test_planted_mistake_fails_a_pin(name):
    with planted(**MUTANTS[name]) as mod:
        assert any(_pins_fail(mod)), name
    assert not any(_pins_fail(H))
