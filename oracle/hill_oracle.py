"""Plain FP64 CPU oracle of the separation-of-variables reference solution.

TEST INFRASTRUCTURE.  Only the tests, the smoke check and the CPU legs of the
benchmark may import this module.  The CUDA library never calls it and shares
no code with it.

What it computes (Bruno & Maas, Sec. 3.1): for a permittivity that does not
depend on x, the exact one-way field u(x, z) = sum_i a_i exp(i alpha_i x)
phi_i(z) (Eq. series_sol), where (phi_i, alpha_i^2) are the eigenpairs of the
Sturm-Liouville problem phi'' + k^2 eps phi = alpha^2 phi (Eq. phi_equation)
and a_i are the projections of the field at x = 0 on the orthonormal
eigenfunctions (Eqs. series_init, sl_expansion).

Readings (the paper discretises the problem with a spectral eigensolver it
does not describe):

  H1  Discretisation: Galerkin on the Fourier modes |n| <= K of the period,
      split by parity about a symmetry point z_c of eps.  Grounded domains
      (Neumann or Dirichlet at z_a, the period [2 z_a - z_b, z_b) of the
      S-WKB mirror, z_c = z_a) keep the even (cosine, n = 0..K) or the odd
      (sine, n = 1..K) modes; periodic media even about z_c keep both.  In the
      orthonormal bases e_0 = 1, e_n = sqrt(2) cos(kappa_n s) and
      e_n = sqrt(2) sin(kappa_n s), s = z - z_c, kappa_n = 2 pi n / L, the
      matrix of phi -> phi'' + k^2 eps phi is
          A_nm = -kappa_n^2 delta_nm + k^2 w_n w_m (eh_|n-m| +- eh_(n+m)) / 2,
      w_0 = 1, w_n = sqrt(2); + for cosines, - for sines, where
      eh_j = <eps cos(kappa_j s)> is the period mean.  It is real symmetric
      and has the eigenpairs of the truncated Hill matrix on that parity.
  H2  eh_j comes from n_q + 1 samples of eps on the half period from z_c,
      s_i = i L / (2 n_q), by the rectangle rule on the whole period (the
      even extension), i.e. a type-1 cosine transform; n_q >= 2 K.
  H3  alpha_i is the principal square root of the eigenvalue: modes with
      alpha_i^2 < 0 decay as exp(-sqrt(-alpha_i^2) x).
  H4  The field is given on the S-WKB grid (grounded: z_a + m dz, m < n_z,
      dz = H / n_z, mirrored onto the period with zero at the top point
      z_b; periodic: n_z points over [z_a, z_b)); z_c is a grid point.  The
      projections are the period means <u e_n> over that grid, which are
      exact for fields band-limited to |n| <= K, and the result is returned
      on the same points.
"""
from __future__ import annotations

import math

import numpy as np

BC_PERIODIC, BC_NEUMANN, BC_DIRICHLET = 0, 1, 2


def period_grid(bc, z_a, z_b, n_z, z_c=None):
    """(L, N, m_c, dz): period length, period points, index of z_c on the
    period grid, grid spacing (reading H4)."""
    if bc == BC_PERIODIC:
        L, N = z_b - z_a, n_z
        dz = L / N
        m_c = int(round((z_c - z_a) / dz))
        if abs(z_a + m_c * dz - z_c) > 1e-9 * dz:
            raise ValueError("the symmetry point must be a grid point")
    else:
        L, N = 2.0 * (z_b - z_a), 2 * n_z
        dz = (z_b - z_a) / n_z
        m_c = n_z
    return L, N, m_c, dz


def parities(bc):
    return {BC_PERIODIC: ("even", "odd"), BC_NEUMANN: ("even",), BC_DIRICHLET: ("odd",)}[bc]


def cosine_coefficients(eps_half, n_out):
    """eh_j, j < n_out, from eps at s_i = i L / (2 n_q), i = 0..n_q
    (reading H2): the mean over the period of the even extension."""
    e = np.asarray(eps_half, float)
    n_q = len(e) - 1
    full = np.concatenate([e, e[n_q - 1:0:-1]])       # eps(s_i), i = 0 .. 2 n_q - 1
    i = np.arange(2 * n_q)
    out = np.empty(n_out)
    for j in range(n_out):
        out[j] = np.mean(full * np.cos(math.pi * j * i / n_q))
    return out


def hill_matrix(k, L, eh, K, parity):
    """A of reading H1 for one parity (size K + 1 for cosines, K for sines)."""
    n = np.arange(0, K + 1) if parity == "even" else np.arange(1, K + 1)
    w = np.where(n == 0, 1.0, math.sqrt(2.0))
    sign = 1.0 if parity == "even" else -1.0
    nm = n[:, None], n[None, :]
    A = k * k * np.outer(w, w) * (eh[np.abs(nm[0] - nm[1])] + sign * eh[nm[0] + nm[1]]) / 2.0
    A[np.diag_indices_from(A)] -= (2.0 * math.pi * n / L) ** 2
    return A, n, w


def field_on_period(u, bc, n_z):
    """The S-WKB mirror of a grounded field onto its period (zero at the top
    point), or the field itself for periodic media."""
    u = np.asarray(u, complex)
    if bc == BC_PERIODIC:
        return u.copy()
    full = np.zeros(2 * n_z, complex)
    sgn = 1.0 if bc == BC_NEUMANN else -1.0
    full[n_z:] = u
    full[n_z - np.arange(1, n_z)] = sgn * u[1:]
    return full


def basis(parity, n, w, N, m_c):
    """e_n at the period points, rows n (exact integer phase (n (i - m_c)) mod N)."""
    ph = (np.outer(n, np.arange(N) - m_c) % N) * (2.0 * math.pi / N)
    return w[:, None] * (np.cos(ph) if parity == "even" else np.sin(ph))


def propagate(k, eps_half, u0, xs, bc, z_a, z_b, K, z_c=None, return_eigs=False):
    """u(x, z_m) for every x in xs (Eq. series_sol), rows in the order of xs,
    on the points of u0.  eps_half: eps at z_c + i L / (2 n_q), i = 0..n_q."""
    n_z = len(u0)
    z_c = z_a if bc != BC_PERIODIC else z_c
    L, N, m_c, _ = period_grid(bc, z_a, z_b, n_z, z_c)
    if len(eps_half) - 1 < 2 * K:
        raise ValueError("need n_q >= 2 K samples of eps on the half period")
    if K >= N // 2:
        raise ValueError("K must be below half the period points")
    eh = cosine_coefficients(eps_half, 2 * K + 1)
    full = field_on_period(u0, bc, n_z)
    out = np.zeros((len(xs), N), complex)
    eigs = {}
    for par in parities(bc):
        A, n, w = hill_matrix(k, L, eh, K, par)
        lam, V = np.linalg.eigh(A)                       # library primitive
        alpha = np.sqrt(lam.astype(complex))              # reading H3
        E = basis(par, n, w, N, m_c)
        uh = E @ full / N                                 # <u e_n> (Eq. sl_expansion)
        a = V.T @ uh                                      # on the eigenfunctions
        for r, x in enumerate(xs):
            out[r] += (V @ (a * np.exp(1j * alpha * x))) @ E    # Eq. series_sol
        eigs[par] = lam
    res = out[:, m_c:m_c + n_z] if bc != BC_PERIODIC else out
    return (res, eigs) if return_eigs else res
