"""Exact / closed-form references used to pin the oracle (test-only).

None of these calls the oracle: each is an independent solution of the
Helmholtz problem (or of the ray equations) in a case where one is known.
"""
from __future__ import annotations

import math

import numpy as np
from scipy import special


def angular_spectrum(u0, k, L, dx_total, n_max, eps0=1.0):
    """Discrete angular-spectrum propagation of a periodic field through a
    homogeneous medium eps0 over range dx_total, keeping |n| <= n_max:
    the exact one-way Helmholtz solution for the band-limited field."""
    N = len(u0)
    n = np.rint(np.fft.fftfreq(N, 1.0 / N)).astype(np.int64)
    kz = 2.0 * math.pi * n / L
    kx = np.sqrt(np.maximum(k * k * eps0 - kz * kz, 0.0))
    H = np.where(np.abs(n) <= n_max, np.exp(1j * kx * dx_total), 0.0)
    return np.fft.ifft(np.fft.fft(u0) * H)


def linear_ray(kappa, s, a, x, eps0=1.0):
    """Closed-form ray of eps = eps0 + a z launched at (0, s) with psi_z =
    kappa: P is conserved, Q = kappa + a x/(2P), z parabolic, residual phase
    r = psi - kappa (z - s) cubic in x, and the s-variations Z_s, Q_s."""
    P = math.sqrt(eps0 + a * s - kappa * kappa)
    z = s + kappa * x / P + a * x * x / (4.0 * P * P)
    Q = kappa + a * x / (2.0 * P)
    r = P * x + a * kappa * x * x / (4.0 * P * P) + a * a * x ** 3 / (12.0 * P ** 3)
    Zs = 1.0 - a * kappa * x / (2.0 * P ** 3) - a * a * x * x / (4.0 * P ** 4)
    Qs = -a * a * x / (4.0 * P ** 3)
    return dict(z=z, Q=Q, r=r, Zs=Zs, Qs=Qs, P=P)


def airy_field(u0, z, k, a, x, zeta):
    """Exact one-way Helmholtz field for eps = 1 + a z (whole line in z).

    Separation of variables gives modes e^{i beta x} Ai(c (zeta - z)) with
    c = (k^2 a)^{1/3} and beta = k sqrt(1 + a zeta) (zeta = turning height).
    The Airy completeness relation gives the mode weights
    A(zeta) = c^2 int u0(z) Ai(c (zeta - z)) dz.  Quadrature: trapezoid on the
    uniform grids z (field samples) and zeta."""
    c = (k * k * a) ** (1.0 / 3.0)
    dz = z[1] - z[0]
    dzeta = zeta[1] - zeta[0]
    out = np.zeros(len(z), dtype=np.complex128)
    beta = k * np.sqrt(1.0 + a * zeta + 0j)
    chunk = 512
    for i0 in range(0, len(zeta), chunk):
        zt = zeta[i0:i0 + chunk]
        Ai = special.airy(c * (zt[:, None] - z[None, :]))[0]
        A = c * c * (Ai @ u0) * dz
        out += (A * np.exp(1j * beta[i0:i0 + chunk] * x)) @ Ai * dzeta
    return out


def hill_one_way(u0, k, L, eps, x, K, n_quad=4096):
    """Separation-of-variables solution (Sec. 3.1, Eqs. series_sol,
    phi_equation, series_init, sl_expansion) for an x-invariant permittivity
    periodic on the period of the field samples u0 (N samples over length L);
    eps is a callable of the offset t in [0, L) from the first sample.

    The Sturm-Liouville problem phi'' + k^2 eps phi = alpha^2 phi with
    periodic conditions is discretised by Fourier-Galerkin on the modes
    |n| <= K (the Hill matrix H_nm = -(2 pi n / L)^2 delta_nm + k^2 eps^_(n-m),
    eps^_j the Fourier coefficients of eps); H is Hermitian, so its
    eigenvectors are orthonormal and the expansion coefficients of u0 are
    plain projections.  Each eigen-mode advances by exp(i alpha x), alpha =
    sqrt(lambda) (decaying for lambda < 0).  Returns u(x) on the same grid."""
    N = len(u0)
    t = L * np.arange(n_quad) / n_quad
    eh = np.fft.fft(eps(t)) / n_quad                      # eps^_j, j mod n_quad
    n = np.arange(-K, K + 1)
    j = (n[:, None] - n[None, :]) % n_quad
    H = k * k * eh[j]
    H[np.diag_indices_from(H)] += -(2.0 * math.pi * n / L) ** 2
    lam, V = np.linalg.eigh(H)
    alpha = np.sqrt(lam.astype(np.complex128))
    uh = np.fft.fft(u0) / N                               # u0 = sum_n uh_n e^{2 pi i n m / N}
    c = V.conj().T @ uh[n % N]
    vh = V @ (c * np.exp(1j * alpha * x))
    out_h = np.zeros(N, dtype=np.complex128)
    out_h[n % N] = vh
    return np.fft.ifft(out_h) * N
