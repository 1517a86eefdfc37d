"""Fields on planes between screens (swkb_propagate_planes) against the
oracle's propagate_planes, the closed-form angular spectrum, and the plain
screen snapshots."""
import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import Oracle, geometry, rel_l2

pytestmark = pytest.mark.gpu

PRECS = [(swkb.SWKB_FP64, 1e-9), (swkb.SWKB_MIXED, 1e-4)]
_cache = {}


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def _oracle_rows(name, pb, planes):
    if name not in _cache:
        _cache[name] = Oracle(pb).propagate_planes(pb.u0, 0, pb.n_screens, planes)
    return _cache[name]


def _rows_close(got, want, tol):
    # every plane's field within tol (rel-L2) of the oracle's
    assert got.shape == want.shape
    return max(rel_l2(g, r) for g, r in zip(got, want)) < tol


@pytest.mark.parametrize("prec,tol", PRECS)
def test_planes_periodic_match_oracle(prec, tol):
    pb = w.config_unit_periodic(n_screens=3)
    want = _oracle_rows("c1", pb, 4)
    got = swkb.Plan(pb, prec, planes=4).propagate_planes(4)
    assert _rows_close(got, want, tol)


@pytest.mark.parametrize("prec,tol", PRECS)
def test_planes_grounded_match_oracle(prec, tol):
    # Neumann ground, top absorber: the inner planes carry no absorber
    pb = w.config_surface_duct_small(n_screens=2)
    want = _oracle_rows("duct", pb, 4)
    got = swkb.Plan(pb, prec, planes=4).propagate_planes(4)
    assert _rows_close(got, want, tol)


@pytest.mark.parametrize("bc", [w.BC_PERIODIC, w.BC_DIRICHLET])
@pytest.mark.parametrize("prec,tol", PRECS)
def test_planes_homogeneous_closed_form(bc, prec, tol):
    from refs import angular_spectrum
    pb = w.config_homogeneous(eps0=1.04, bc=bc, ray_stride=2, rk4_steps=6, n_screens=2)
    P = 3
    got = swkb.Plan(pb, prec, planes=P).propagate_planes(P)
    g = geometry(pb)
    n = pb.n_z
    for q in range(pb.n_screens):
        for j in range(1, P + 1):
            d = (q + j / P) * pb.dx
            if bc == w.BC_PERIODIC:
                ref = angular_spectrum(pb.u0, pb.k, g.L, d, g.n_max, 1.04)
            else:
                full = np.zeros(2 * n, complex)
                full[n:] = pb.u0
                full[n - np.arange(1, n)] = -pb.u0[1:]
                ref = angular_spectrum(full, pb.k, g.L, d, g.n_max, 1.04)[n:]
            assert rel_l2(got[q * P + j - 1], ref) < tol


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_last_plane_of_each_screen_is_the_snapshot(prec):
    pb = w.config_surface_duct_small(n_screens=3)
    plan = swkb.Plan(pb, prec, planes=4)
    rows = plan.propagate_planes(4)
    snaps = plan.propagate(snapshot_every=1)
    assert np.array_equal(rows[3::4], snaps)
    # one plane per screen needs no plane buffers and gives the snapshots too
    assert np.array_equal(swkb.Plan(pb, prec).propagate_planes(1), snaps)


def test_planes_device_pointers_equal_host():
    torch = pytest.importorskip("torch")
    pb = w.config_unit_periodic(n_screens=2)
    plan = swkb.Plan(pb, swkb.SWKB_MIXED, planes=2)
    host = plan.propagate_planes(2)
    u0 = torch.from_numpy(pb.u0).cuda()
    out = torch.zeros((4, pb.n_z), dtype=torch.complex128, device="cuda")
    plan.propagate_planes_device(2, u0.data_ptr(), out.data_ptr())
    torch.cuda.synchronize()
    assert np.array_equal(out.cpu().numpy(), host)


def test_planes_arguments_checked():
    pb = w.config_unit_periodic(n_screens=1)            # rk4_steps 8
    with pytest.raises(swkb.SwkbError) as e:
        swkb.Plan(pb, swkb.SWKB_MIXED, planes=3)       # does not divide 8
    assert e.value.status == swkb.SWKB_ERR_INVALID_ARG
    plan = swkb.Plan(pb, swkb.SWKB_MIXED, planes=2)
    for bad in (0, 3, 4):                               # 4 divides 8 but exceeds the buffers
        with pytest.raises(swkb.SwkbError) as e:
            plan.propagate_planes(bad)
        assert e.value.status == swkb.SWKB_ERR_INVALID_ARG
