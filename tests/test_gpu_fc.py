"""Patch-wise Fourier-continuation screens (Sec. 2.2) on the GPU, through the
C ABI, against the continuation oracle (oracle/fc_oracle.py).

Tolerances: FP64 plans max |gpu - oracle| <= 1e-10 of the field's max (same
arithmetic, different summation order); mixed plans (FP32 rays and sum, FP64
continuation and DFT) <= 1e-4."""
import math

import numpy as np
import pytest

import fc_pins as P
from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w

pytestmark = pytest.mark.gpu
pytest.importorskip("mpmath")

from oracle.fc_oracle import FCOracle  # noqa: E402

FP64_TOL = 1e-10
MIXED_TOL = 1e-4


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _err(got, want):
    return float(np.max(np.abs(got - want)) / np.max(np.abs(want)))


def lens(n_screens=2, ray_stride=1, P_=3, n_pat=144, n_ov=48, zc=52.0, tilt=6.0, cols=1):
    H = ((P_ - 1) * (n_pat - n_ov) + n_pat) * P.STEP
    pb = P.open_problem(n_pat, n_ov, P_, zc, tilt, 5.0, medium=w.f_gaussian(0.01, 0.01, zc=H / 2),
                        n_screens=n_screens, rk4_steps=8, ray_stride=ray_stride)
    if cols > 1:
        # range-dependent: the lens strengthens linearly between two columns
        prof = pb.profile
        f2 = w.f_gaussian(0.02, 0.01, zc=H / 2)
        e2, ez2, ezz2 = f2(prof.nodes())
        prof = w.Profile(np.array([0.0, 2 * pb.dx]), prof.z0, prof.dz,
                         np.vstack([prof.eps, e2]), np.vstack([prof.eps_z, ez2]),
                         np.vstack([prof.eps_zz, ezz2]))
        pb = pb.with_(profile=prof)
    return pb


CASES = {
    "lens-3x144": lambda: lens(),
    "lens-R2": lambda: lens(ray_stride=2, P_=4, n_pat=160, n_ov=48),
    "lens-1-patch": lambda: lens(P_=1, n_pat=240, n_ov=48, zc=40.0, n_screens=3),
    "lens-range-dependent": lambda: lens(cols=2, n_screens=3),
    "homogeneous-6x120": lambda: P.open_problem(120, 40, 6, 90.0, -7.0, 5.0, n_screens=2),
    # the smallest accepted patch (16 points, 8 shared) and the longest
    # continued period (N_p = 2048, one patch)
    "edge-min-patch": lambda: P.open_problem(16, 8, 7, 32 * P.STEP, 0.0, 1.0, n_screens=1),
    "edge-max-period": lambda: P.open_problem(2023, 500, 1, 1011 * P.STEP, 5.0, 3.0,
                                              n_screens=1),
}

_oracle = {}


def oracle_field(name):
    if name not in _oracle:
        pb = CASES[name]()
        _oracle[name] = FCOracle(pb).propagate(pb.u0)
    return _oracle[name]


@pytest.mark.parametrize("name", sorted(CASES))
def test_fp64_matches_oracle(name):
    pb = CASES[name]()
    plan = swkb.Plan(pb, precision=swkb.SWKB_FP64)
    assert plan.info.fc_patches == (pb.n_z - pb.fc_patch) // (pb.fc_patch - pb.fc_overlap) + 1
    assert plan.info.fc_period_points == pb.fc_patch + 25
    got = plan.propagate()
    assert _err(got, oracle_field(name)) <= FP64_TOL


@pytest.mark.parametrize("name", sorted(CASES))
def test_mixed_matches_oracle(name):
    pb = CASES[name]()
    got = swkb.Plan(pb, precision=swkb.SWKB_MIXED).propagate()
    assert _err(got, oracle_field(name)) <= MIXED_TOL


def test_modes_and_rays_match_the_oracle_mode_set():
    pb = lens()
    o = FCOracle(pb)
    info = swkb.Plan(pb).info
    assert info.n_max == o.n_max and info.n_ghost == o.G
    assert info.n_fft == (pb.n_z + 63) // 64 * 64
    assert info.n_rays_total == info.n_fft // pb.ray_stride + 2 * o.G
    assert abs(info.period - o.Lp) < 1e-12 * o.Lp


def test_snapshots_and_resume_match_one_call():
    pb = lens(n_screens=4)
    plan = swkb.Plan(pb, precision=swkb.SWKB_FP64)
    whole = plan.propagate()
    snaps = plan.propagate(snapshot_every=2)
    assert np.array_equal(snaps[-1], whole)
    half = plan.propagate(n_screens=2)
    resumed = plan.propagate(u0=half, q0=2, n_screens=2)
    assert np.array_equal(resumed, whole)


def test_homogeneous_against_angular_spectrum():
    """Physics through the GPU: one screen in eps = 1 against the exact
    propagator (the oracle's pin, < 2e-6 with 48-point overlaps)."""
    pb = P.open_problem(144, 48, 3, (144 - 24) * P.STEP, 8.0, 5.0)
    got = swkb.Plan(pb, precision=swkb.SWKB_FP64).propagate()
    assert _err(got, P.angular_spectrum(pb.u0, pb.dx)) < 2e-6


@pytest.mark.parametrize("kw,msg", [
    (dict(fc_patch=80, fc_overlap=16, n_z=300), "tile"),        # patches do not tile n_z
    (dict(fc_patch=30, fc_overlap=16, n_z=272), "tile"),        # ramps would overlap
    (dict(fc_patch=2100, fc_overlap=64, n_z=2100), "2048"),     # continued period too long
])
def test_invalid_layouts_are_refused(kw, msg):
    pb = P.open_problem(144, 48, 3, 50.0, 0.0, 5.0)
    n_z = kw.pop("n_z")
    H = n_z * P.STEP
    pb = pb.with_(n_z=n_z, z_b=H, u0=np.zeros(n_z, dtype=np.complex128), **kw)
    with pytest.raises(swkb.SwkbError) as e:
        swkb.Plan(pb)
    assert e.value.status == swkb.SWKB_ERR_INVALID_ARG
    assert msg in str(e.value)


def test_absorber_is_refused():
    with pytest.raises(swkb.SwkbError):
        swkb.Plan(lens().with_(absorber_frac=0.1))


@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)])
def test_planes_match_oracle(prec, tol):
    """Fields on 4 planes per screen over 2 screens (range-dependent lens:
    the planes' stage columns differ), against the oracle's planes; the last
    plane of each screen equals the plain propagation's screen field."""
    pb = lens(cols=2, n_screens=2)
    want = FCOracle(pb).propagate_planes(pb.u0, 0, 2, 4)
    plan = swkb.Plan(pb, precision=prec, planes=4)
    got = plan.propagate_planes(4)
    assert got.shape == want.shape
    assert np.max(np.abs(got - want)) <= tol * np.max(np.abs(want))
    assert np.array_equal(got[-1], plan.propagate())


@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)])
def test_open_lens_full_size_sampled_against_oracle(prec, tol):
    """The bench's patch-wise workload at full size (N_z = 131072, 188
    patches, R = 8, the launch shapes bench.py uses): screens 0 and 1 on the
    GPU, sampled points of each against the oracle's screen_points, the
    second screen started from the GPU's own first-screen field."""
    pb = w.config_open_lens()
    plan = swkb.Plan(pb, prec)
    f1 = plan.propagate(n_screens=1)
    f2 = plan.propagate(u0=f1, q0=1, n_screens=1)
    o = FCOracle(pb)
    rng = np.random.default_rng(17)
    strong = np.flatnonzero(np.abs(f1) > 0.05 * np.abs(f1).max())
    overlap = np.array([int(o.patches.start[p]) + pb.fc_overlap // 2
                        for p in range(1, o.patches.P)])
    overlap = overlap[np.abs(f1[overlap]) > 1e-3 * np.abs(f1).max()]
    ms = np.unique(np.concatenate([rng.choice(strong, 10, replace=False), overlap[:4]]))
    for q, u_in, got in ((0, pb.u0, f1), (1, f1, f2)):
        want = o.screen_points(u_in, q, ms)
        assert np.max(np.abs(got[ms] - want)) <= tol * np.max(np.abs(got))


def test_plans_of_different_sizes_coexist():
    """The kernels' shared-memory limit is process-wide: creating a plan with
    a shorter continued period and smaller tiles after a larger one must not
    break the larger plan's launches (both FP64: the largest staging)."""
    big = lens(ray_stride=1, P_=2, n_pat=1600, n_ov=200, zc=300.0, n_screens=1)
    small = lens(n_screens=1)
    p_big = swkb.Plan(big, precision=swkb.SWKB_FP64)
    first = p_big.propagate()
    p_small = swkb.Plan(small, precision=swkb.SWKB_FP64)
    p_small.propagate()
    assert np.array_equal(p_big.propagate(), first)
