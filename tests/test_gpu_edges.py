"""Edge cases of the GPU path through the C ABI: empty runs, degenerate mode
sets, a zero field, and the smallest and largest FFT lengths a plan accepts.

Homogeneous media have a closed form (the discrete angular spectrum over the
kept modes), so the size extremes are checked against it at every grid point
without running the oracle at 2^20 points."""
import math

import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import Oracle, geometry, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-4
PRECS = [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)]


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _angular_ref(pb, eps0):
    from refs import angular_spectrum
    g = geometry(pb)
    if pb.bc == w.BC_PERIODIC:
        return angular_spectrum(pb.u0, pb.k, g.L, pb.dx * pb.n_screens, g.n_max, eps0)
    sg = 1.0 if pb.bc == w.BC_NEUMANN else -1.0
    n = pb.n_z
    full = np.zeros(2 * n, complex)
    full[n:] = pb.u0
    full[n - np.arange(1, n)] = sg * pb.u0[1:]
    return angular_spectrum(full, pb.k, g.L, pb.dx * pb.n_screens, g.n_max, eps0)[n:]


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_zero_screens_is_the_identity(prec):
    torch = pytest.importorskip("torch")
    pb = w.config_unit_periodic()
    plan = swkb.Plan(pb, prec)
    got = plan.propagate(n_screens=0)
    assert np.array_equal(got, pb.u0)
    u0 = torch.from_numpy(pb.u0).cuda()
    out = torch.zeros_like(u0)
    plan.propagate_device(u0.data_ptr(), out.data_ptr(), n_screens=0)
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), pb.u0)


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_zero_field_stays_zero(prec):
    pb = w.config_surface_duct_small(n_screens=2)
    pb = pb.with_(u0=np.zeros_like(pb.u0))
    got = swkb.Plan(pb, prec).propagate()
    assert np.count_nonzero(got) == 0


@pytest.mark.parametrize("grounded", [False, True])
@pytest.mark.parametrize("prec,tol", PRECS)
def test_single_kept_mode(prec, tol, grounded):
    # theta_max below the first mode's angle: n_max = 0, one plane wave
    if grounded:
        pb = w.config_surface_duct_small(n_screens=2).with_(theta_max=math.radians(0.02))
    else:
        pb = w.config_gaussian_medium(n_screens=2).with_(theta_max=math.radians(0.5))
    g = geometry(pb)
    assert g.n_max == 0 and g.M == 1
    want = Oracle(pb).propagate(pb.u0)
    got = swkb.Plan(pb, prec).propagate()
    assert rel_l2(got, want) < tol


@pytest.mark.parametrize("prec,tol", PRECS)
def test_smallest_fft_length(prec, tol):
    pb = w.config_homogeneous(eps0=1.05, n_z=64, height=32.0, ray_stride=1, rk4_steps=3)
    assert geometry(pb).N == 64
    got = swkb.Plan(pb, prec).propagate()
    assert rel_l2(got, _angular_ref(pb, 1.05)) < tol


@pytest.mark.parametrize("bc,n_z", [(w.BC_PERIODIC, 1 << 20), (w.BC_NEUMANN, 1 << 19)])
@pytest.mark.parametrize("prec,tol", PRECS)
def test_largest_fft_length(bc, n_z, prec, tol):
    pb = w.config_homogeneous(eps0=1.02, n_z=n_z, height=32.0, ray_stride=64, rk4_steps=2,
                              bc=bc, n_screens=2, theta_deg=20.0)
    assert geometry(pb).N == 1 << 20
    got = swkb.Plan(pb, prec).propagate()
    assert rel_l2(got, _angular_ref(pb, 1.02)) < tol


def test_fft_length_limits_rejected():
    for n_z, bc in ((1 << 21, w.BC_PERIODIC), (1 << 20, w.BC_NEUMANN), (32, w.BC_PERIODIC),
                    (16, w.BC_NEUMANN), (3000, w.BC_PERIODIC)):
        pb = w.config_homogeneous(n_z=n_z, bc=bc, ray_stride=1)
        with pytest.raises(swkb.SwkbError) as e:
            swkb.Plan(pb, swkb.SWKB_MIXED)
        assert e.value.status == swkb.SWKB_ERR_INVALID_ARG
