"""The GPU separation-of-variables path (swkb_sym_eig, swkb_hill_propagate)
against the oracle (oracle/hill_oracle.py, LAPACK eigh) and against the
invariants of a symmetric eigen-decomposition.

Tolerances.  The eigenvalues of both sides carry errors of a few units of
FP64 rounding times ||A|| (Jacobi and Householder-QR are both backward
stable), so a mode's alpha = sqrt(lambda) differs by about
c eps_mach ||A|| / (2 alpha), ||A|| ~ k^2 eps and alpha ~ k: the phase
alpha x then differs by about c eps_mach k x / 2.  The field bound used here
is 1e-11 + 32 eps_mach k x (c = 64): 1e-10 at x = 300 m and k = 2 pi / 5 cm,
1.8e-7 at 200 km."""
import math

import numpy as np
import pytest

from oracle import hill_oracle as H
from oracle.swkb_oracle import rel_l2
from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w

pytestmark = pytest.mark.gpu

EPS = np.finfo(float).eps


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def field_tol(k, x):
    return 1e-11 + 32.0 * EPS * k * x


def _check_eig(A, lam, V, tol=1e-13):
    """Eigenvalues against LAPACK, residual and orthonormality of the rows."""
    A = 0.5 * (A + A.T)
    nrm = max(np.linalg.norm(A, 2), 1e-300)
    ref = np.linalg.eigvalsh(A)
    assert np.max(np.abs(np.sort(lam) - ref)) <= tol * nrm * max(1, len(lam)) ** 0.5
    assert np.max(np.abs(V @ A - lam[:, None] * V)) <= 10 * tol * nrm * len(lam) ** 0.5
    assert np.max(np.abs(V @ V.T - np.eye(len(lam)))) <= 10 * tol * len(lam) ** 0.5


@pytest.mark.parametrize("n", [1, 2, 3, 17, 64, 255])
def test_sym_eig_random(n):
    rng = np.random.default_rng(n)
    A = rng.standard_normal((3, n, n))
    A = A + A.transpose(0, 2, 1)
    lam, V, sweeps = swkb.swkb_sym_eig(A)
    assert sweeps <= 15
    for b in range(3):
        _check_eig(A[b], lam[b], V[b])


def test_sym_eig_degenerate_and_diagonal():
    rng = np.random.default_rng(5)
    Q, _ = np.linalg.qr(rng.standard_normal((40, 40)))
    d = np.repeat([-3.0, 0.5, 0.5 + 1e-13, 2.0], 10)
    A = Q @ np.diag(d) @ Q.T
    lam, V, _ = swkb.swkb_sym_eig(A)
    _check_eig(A, lam, V)
    D = np.diag(np.arange(9.0))
    lam, V, sweeps = swkb.swkb_sym_eig(D)
    assert sweeps == 0 and np.array_equal(lam, np.arange(9.0)) and np.array_equal(V, np.eye(9))


def test_sym_eig_uses_the_symmetric_part_and_keeps_the_input():
    rng = np.random.default_rng(6)
    A = rng.standard_normal((30, 30))
    keep = A.copy()
    lam, V, _ = swkb.swkb_sym_eig(A)
    _check_eig(A, lam, V)
    assert np.array_equal(A, keep)


def test_sym_eig_device_pointers():
    import torch
    rng = np.random.default_rng(8)
    A = rng.standard_normal((4, 33, 33))
    A = A + A.transpose(0, 2, 1)
    lam_h, V_h, _ = swkb.swkb_sym_eig(A)
    a = torch.from_numpy(A).cuda()
    lam = torch.empty((4, 33), dtype=torch.float64, device="cuda")
    vec = torch.empty((4, 33, 33), dtype=torch.float64, device="cuda")
    s = torch.cuda.Stream()
    swkb.swkb_sym_eig_device(4, 33, a.data_ptr(), lam.data_ptr(), vec.data_ptr(), s.cuda_stream)
    assert np.array_equal(lam.cpu().numpy(), lam_h) and np.array_equal(vec.cpu().numpy(), V_h)


@pytest.mark.parametrize("bad", ["n0", "batch0", "nan"])
def test_sym_eig_rejects(bad):
    A = np.eye(4)
    if bad == "nan":
        A[1, 2] = np.nan
    with pytest.raises((swkb.SwkbError, ValueError)) as e:
        if bad == "n0":
            swkb.swkb_sym_eig(np.zeros((2, 0, 0)))
        elif bad == "batch0":
            swkb.swkb_sym_eig(np.zeros((0, 3, 3)))
        else:
            swkb.swkb_sym_eig(A)
    if isinstance(e.value, swkb.SwkbError):
        assert e.value.status == swkb.SWKB_ERR_INVALID_ARG


# --------------------------------------------------------------------------
# swkb_hill_propagate against the oracle
# --------------------------------------------------------------------------
def _duct(seed=12, n_z=1024, height=25.0, bc=w.BC_NEUMANN):
    pb = w.config_surface_duct_small(seed=seed, n_z=n_z, height=height)
    f = w.f_trilinear_duct(pb.meta["z_t"], pb.meta["g_d"])
    u0 = pb.u0 if bc == w.BC_NEUMANN else pb.u0 * np.sin(math.pi * np.arange(n_z) / n_z)
    return pb, (lambda z: f(np.asarray(z))[0]), u0


def _sorted_eigs(eigs, bc, K):
    pars = H.parities(bc)
    return [np.sort(eigs[p]) for p in pars]


def _gpu_blocks(lam, bc, K):
    if bc == w.BC_PERIODIC:
        return [np.sort(lam[:K + 1]), np.sort(lam[K + 1:])]
    return [np.sort(lam)]


@pytest.mark.parametrize("bc", [w.BC_NEUMANN, w.BC_DIRICHLET])
def test_grounded_duct_matches_oracle(bc):
    pb, eps, u0 = _duct(bc=bc)
    Hh, K = pb.z_b - pb.z_a, 160
    n_q = 2 * K + 7
    s = np.arange(n_q + 1) * Hh / n_q
    xs = [0.0, 35.0, 300.0]
    want, eigs = H.propagate(pb.k, eps(s), u0, xs, bc, pb.z_a, pb.z_b, K, return_eigs=True)
    d = swkb.hill_desc(bc, pb.z_a, pb.z_b, pb.n_z, K, n_q)
    got, lam = swkb.swkb_hill_propagate(d, [pb.k], eps(s)[None], u0[None], xs, eigenvalues=True)
    for r, x in enumerate(xs):
        assert rel_l2(got[0, r], want[r]) < field_tol(pb.k, x), x
    for g, o in zip(_gpu_blocks(lam[0], bc, K), _sorted_eigs(eigs, bc, K)):
        assert np.max(np.abs(g - o)) < 1e-13 * np.max(np.abs(o)) * K ** 0.5


def test_periodic_symmetric_layer_matches_oracle():
    k, L, n_z, K = 2.0 * math.pi, 64.0, 512, 100
    n_q = 2 * K
    f = lambda t: 1.0 + 0.02 * np.exp(-0.01 * (t - L / 2) ** 2)
    s = L / 2 + np.arange(n_q + 1) * L / (2 * n_q)
    z = np.arange(n_z) * L / n_z
    u0 = np.exp(-((z - 20.0) / 3.0) ** 2) * np.exp(1j * 0.3 * k * z)
    xs = [5.0, 40.0]
    want, eigs = H.propagate(k, f(s), u0, xs, H.BC_PERIODIC, 0.0, L, K, z_c=L / 2,
                             return_eigs=True)
    d = swkb.hill_desc(w.BC_PERIODIC, 0.0, L, n_z, K, n_q, z_sym=L / 2)
    got, lam = swkb.swkb_hill_propagate(d, [k], f(s)[None], u0[None], xs, eigenvalues=True)
    for r, x in enumerate(xs):
        assert rel_l2(got[0, r], want[r]) < field_tol(k, x)
    for g, o in zip(_gpu_blocks(lam[0], w.BC_PERIODIC, K), _sorted_eigs(eigs, w.BC_PERIODIC, K)):
        assert np.max(np.abs(g - o)) < 1e-13 * np.max(np.abs(o)) * K ** 0.5


def test_batch_of_different_media_and_wavenumbers():
    """Three ducts (own seeds, so own duct heights and gradients) at three
    wavenumbers in one call: each equals its own oracle run."""
    Hh, n_z, K = 25.0, 512, 96
    n_q = 2 * K
    ks, epss, u0s, wants = [], [], [], []
    for seed, scale in ((1, 1.0), (2, 0.8), (3, 0.6)):
        pb, eps, u0 = _duct(seed=seed, n_z=n_z, height=Hh)
        k = pb.k * scale
        s = np.arange(n_q + 1) * Hh / n_q
        ks.append(k)
        epss.append(eps(s))
        u0s.append(u0)
        wants.append(H.propagate(k, eps(s), u0, [120.0], H.BC_NEUMANN, 0.0, Hh, K)[0])
    d = swkb.hill_desc(w.BC_NEUMANN, 0.0, Hh, n_z, K, n_q)
    got = swkb.swkb_hill_propagate(d, ks, np.array(epss), np.array(u0s), [120.0])
    for b in range(3):
        assert rel_l2(got[b, 0], wants[b]) < field_tol(ks[b], 120.0), b


@pytest.mark.parametrize("K", [1, 2, 5])
def test_few_modes(K):
    pb, eps, u0 = _duct(n_z=64, height=2.0)
    n_q = 2 * K
    s = np.arange(n_q + 1) * 2.0 / n_q
    want = H.propagate(pb.k, eps(s), u0, [3.0], H.BC_NEUMANN, 0.0, 2.0, K)[0]
    d = swkb.hill_desc(w.BC_NEUMANN, 0.0, 2.0, 64, K, n_q)
    got = swkb.swkb_hill_propagate(d, [pb.k], eps(s)[None], u0[None], [3.0])
    assert rel_l2(got[0, 0], want) < field_tol(pb.k, 3.0)


def test_device_pointers_equal_host_buffers():
    import torch
    pb, eps, u0 = _duct(n_z=512, height=25.0)
    K, n_q = 64, 128
    s = np.arange(n_q + 1) * 25.0 / n_q
    d = swkb.hill_desc(w.BC_NEUMANN, 0.0, 25.0, 512, K, n_q)
    xs = [10.0, 50.0]
    host, lam_h = swkb.swkb_hill_propagate(d, [pb.k], eps(s)[None], u0[None], xs,
                                           eigenvalues=True)
    e = torch.from_numpy(eps(s)[None].copy()).cuda()
    u = torch.from_numpy(u0[None].copy()).cuda()
    out = torch.empty((1, 2, 512), dtype=torch.complex128, device="cuda")
    lam = torch.empty((1, K + 1), dtype=torch.float64, device="cuda")
    st = torch.cuda.Stream()
    swkb.swkb_hill_propagate_device(d, [pb.k], e.data_ptr(), u.data_ptr(), xs, out.data_ptr(),
                                    lam.data_ptr(), st.cuda_stream)
    assert np.array_equal(out.cpu().numpy(), host)
    assert np.array_equal(lam.cpu().numpy(), lam_h)


@pytest.mark.parametrize("bad", ["K0", "Kbig", "nq", "zsym", "k", "x", "nan", "bc"])
def test_hill_rejects(bad):
    Hh, n_z, K, n_q = 10.0, 128, 8, 16
    kw = dict(bc=w.BC_NEUMANN, z_a=0.0, z_b=Hh, n_z=n_z, K=K, n_q=n_q)
    k, x = [10.0], [1.0]
    eps = np.ones((1, n_q + 1))
    if bad == "K0":
        kw["K"] = 0
    elif bad == "Kbig":
        kw.update(K=n_z, n_q=2 * n_z)
        eps = np.ones((1, 2 * n_z + 1))
    elif bad == "nq":
        kw["n_q"] = 2 * K - 1
        eps = np.ones((1, 2 * K))
    elif bad == "zsym":
        kw.update(bc=w.BC_PERIODIC, z_sym=0.3 * Hh / n_z)
    elif bad == "k":
        k = [0.0]
    elif bad == "x":
        x = [-1.0]
    elif bad == "nan":
        eps[0, 3] = np.nan
    elif bad == "bc":
        kw["bc"] = 7
    d = swkb.hill_desc(**kw)
    with pytest.raises(swkb.SwkbError) as e:
        swkb.swkb_hill_propagate(d, k, eps, np.ones((1, n_z), complex), x)
    assert e.value.status == swkb.SWKB_ERR_INVALID_ARG


def test_full_size_duct_2km():
    """The 16384-point surface duct over its 2 km separation-of-variables
    check (K = 640 cosines, n_q = 32768) against the oracle."""
    pb = w.config_surface_duct(n_screens=40, range_m=2000.0).with_(absorber_frac=0.0)
    f = w.f_trilinear_duct(pb.meta["z_t"], pb.meta["g_d"])
    Hh, K, n_q = pb.z_b - pb.z_a, 640, 1 << 15
    s = np.arange(n_q + 1) * Hh / n_q
    e = f(s)[0]
    want = H.propagate(pb.k, e, pb.u0, [2000.0], H.BC_NEUMANN, pb.z_a, pb.z_b, K)[0]
    d = swkb.hill_desc(w.BC_NEUMANN, pb.z_a, pb.z_b, pb.n_z, K, n_q)
    got = swkb.swkb_hill_propagate(d, [pb.k], e[None], pb.u0[None], [2000.0])
    assert rel_l2(got[0, 0], want) < field_tol(pb.k, 2000.0)


def test_gaussian_duct_200km():
    """Like the paper's second example: the 400 m periodic domain with a
    narrow Gaussian duct at its centre, K = 220, 200 km."""
    pb = w.config_gaussian_duct_200km()
    a, b = pb.meta["a"], pb.meta["b"]
    L, K, n_q = pb.z_b - pb.z_a, pb.n_max + 100, 4096
    s = np.arange(n_q + 1) * L / (2 * n_q)            # from the centre z = 0
    e = 1.0 + a * np.exp(-b * s ** 2)
    want = H.propagate(pb.k, e, pb.u0, [200_000.0], H.BC_PERIODIC, pb.z_a, pb.z_b, K, z_c=0.0)
    d = swkb.hill_desc(w.BC_PERIODIC, pb.z_a, pb.z_b, pb.n_z, K, n_q, z_sym=0.0)
    got = swkb.swkb_hill_propagate(d, [pb.k], e[None], pb.u0[None], [200_000.0])
    assert rel_l2(got[0, 0], want[0]) < field_tol(pb.k, 200_000.0)


def test_batch_of_periodic_layers_at_several_ranges():
    """Two symmetric layers (both parities, so four matrices) at two ranges
    in one call: each (problem, range) equals its own oracle run."""
    k, L, n_z, K = 2.0 * math.pi, 64.0, 512, 80
    n_q = 2 * K
    s = L / 2 + np.arange(n_q + 1) * L / (2 * n_q)
    z = np.arange(n_z) * L / n_z
    xs = [7.0, 31.0]
    ks, epss, u0s = [], [], []
    for b, (a, w0) in enumerate(((0.02, 3.0), (-0.015, 4.5))):
        f = lambda t, a=a: 1.0 + a * np.exp(-0.01 * (t - L / 2) ** 2)
        ks.append(k * (1.0 + 0.1 * b))
        epss.append(f(s))
        u0s.append(np.exp(-((z - 24.0 - 5 * b) / w0) ** 2) * np.exp(1j * 0.2 * k * z))
    d = swkb.hill_desc(w.BC_PERIODIC, 0.0, L, n_z, K, n_q, z_sym=L / 2)
    got = swkb.swkb_hill_propagate(d, ks, np.array(epss), np.array(u0s), xs)
    for b in range(2):
        want = H.propagate(ks[b], epss[b], u0s[b], xs, H.BC_PERIODIC, 0.0, L, K, z_c=L / 2)
        for r, x in enumerate(xs):
            assert rel_l2(got[b, r], want[r]) < field_tol(ks[b], x), (b, x)


def test_rotation_log_growth(monkeypatch):
    """The rotation log starts with room for one sweep (test knob) and grows
    at sweeps 1, 2 and 4: the fields equal those of the default capacity bit
    for bit."""
    pb, eps, u0 = _duct(n_z=512, height=25.0)
    K, n_q = 96, 192
    s = np.arange(n_q + 1) * 25.0 / n_q
    d = swkb.hill_desc(w.BC_NEUMANN, 0.0, 25.0, 512, K, n_q)
    want = swkb.swkb_hill_propagate(d, [pb.k], eps(s)[None], u0[None], [80.0])
    monkeypatch.setenv("SWKB_HILL_LOG_SWEEPS", "1")
    got = swkb.swkb_hill_propagate(d, [pb.k], eps(s)[None], u0[None], [80.0])
    assert np.array_equal(got, want)
