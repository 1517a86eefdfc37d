"""GPU path (libswkb.so through the C ABI) against the CPU oracle.

Tolerances: FP64 path rel-L2 <= 1e-9 on the field (elementwise <= 1e-9 of the
field's max on intermediates); mixed FP32/FP64 path rel-L2 <= 1e-4."""
import math

import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import Oracle, geometry, rel_l2

pytestmark = pytest.mark.gpu

FP64_TOL = 1e-9
MIXED_TOL = 1e-4


def gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    gpu()


def _oracle_cache():
    cache = {}

    def get(name, fn):
        if name not in cache:
            cache[name] = fn()
        return cache[name]
    return get


_cache = _oracle_cache()


def c1_oracle():
    pb = w.config_unit_periodic()
    return _cache("c1", lambda: Oracle(pb).propagate(pb.u0))


def duct_small():
    return w.config_surface_duct_small()


def duct_small_oracle():
    pb = duct_small()
    return _cache("duct", lambda: Oracle(pb).propagate(pb.u0))


@pytest.mark.parametrize("name", ["unit-periodic", "duct-small", "homog-neumann"])
def test_plan_geometry_matches_oracle(name):
    pb = {"unit-periodic": w.config_unit_periodic, "duct-small": duct_small,
          "homog-neumann": lambda: w.config_homogeneous(bc=w.BC_NEUMANN, ray_stride=2)}[name]()
    g = geometry(pb)
    info = swkb.Plan(pb).info
    assert (info.n_fft, info.n_max, info.n_modes, info.n_rays, info.n_ghost,
            info.n_rays_total) == (g.N, g.n_max, g.M, g.N_r, g.G, g.NRT)


@pytest.mark.parametrize("q", [0, 5])
def test_debug_screen_fp64_intermediates(q):
    pb = w.config_unit_periodic()
    o = Oracle(pb)
    rng = np.random.default_rng(q)
    u = o.extend(pb.u0) * (1 + 0.1 * rng.standard_normal(o.g.N))
    want_u, want_c, rays = o.screen(u, q, keep_rays=True)
    got = swkb.Plan(pb).debug_screen(q, u)
    assert np.max(np.abs(got["c"] - want_c)) <= 1e-13 * np.max(np.abs(want_c))
    delta = (rays["z"] - o.g.z_lo) / o.g.dz
    # the two sides evaluate eps_zz with different rounding (the oracle's
    # Hermite basis cancels terms of size eps / h^2): 1e-10 on the ray data
    assert np.max(np.abs(got["delta"] - delta)) < 1e-9
    assert np.max(np.abs(got["r"] - rays["r"])) < 1e-10
    assert np.max(np.abs(got["a"] - rays["a"])) < 1e-10
    assert rel_l2(got["u_next"], want_u) < FP64_TOL


@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, 1e-9), (swkb.SWKB_MIXED, 1e-4)])
def test_debug_screen_grounded_mirrored_rays(prec, tol):
    """Grounded plans march n >= 0 only; mode -n's rays are mirror images.
    All modes' landings, phases and amplitudes still match the oracle's own
    rays (ray 0 of a mirrored family has no partner and is NaN)."""
    pb = duct_small()
    o = Oracle(pb)
    u = o.extend(pb.u0)
    want_u, want_c, rays = o.screen(u, 3, keep_rays=True)
    got = swkb.Plan(pb, prec).debug_screen(3, u)
    delta = (rays["z"] - o.g.z_lo) / o.g.dz
    neg = o.n < 0
    assert np.all(np.isnan(got["delta"][neg, 0])) and not np.any(np.isnan(got["delta"][~neg]))
    sl = (slice(None), slice(1, None))
    # FP64: rounding only.  FP32: landings to 1e-3 grid cells (1.2e-6 m), phase
    # to 1e-4 rad, amplitude factors to 1e-5.
    tol_d, tol_phase, tol_a = (1e-9, 1e-8, 1e-10) if prec == swkb.SWKB_FP64 else (1e-3, 1e-4, 1e-5)
    assert np.max(np.abs(got["delta"][sl] - delta[sl])) < tol_d
    assert np.max(np.abs(got["r"][sl] - rays["r"][sl])) * pb.k < tol_phase
    assert np.max(np.abs(got["a"][sl] - rays["a"][sl])) < tol_a
    assert rel_l2(got["u_next"], o.project(want_u)) < tol


def test_debug_screen_mixed_intermediates():
    pb = w.config_unit_periodic()
    o = Oracle(pb)
    u = o.extend(pb.u0)
    want_u, want_c, rays = o.screen(u, 5, keep_rays=True)
    got = swkb.Plan(pb, swkb.SWKB_MIXED).debug_screen(5, u)
    assert np.max(np.abs(got["c"] - want_c)) <= 1e-6 * np.max(np.abs(want_c))
    delta = (rays["z"] - o.g.z_lo) / o.g.dz
    assert np.max(np.abs(got["delta"] - delta)) < 1e-4
    # residual phase in turns: k r / (2 pi) within 1e-5 turn
    assert np.max(np.abs(got["r"] - rays["r"])) * pb.k / (2 * math.pi) < 1e-5
    assert np.max(np.abs(got["a"] - rays["a"])) < 1e-5
    assert rel_l2(got["u_next"], want_u) < MIXED_TOL


def test_unit_periodic_fp64_parity():
    pb = w.config_unit_periodic()
    got = swkb.Plan(pb).propagate()
    assert rel_l2(got, c1_oracle()) < FP64_TOL


def test_unit_periodic_mixed_parity():
    pb = w.config_unit_periodic()
    got = swkb.Plan(pb, swkb.SWKB_MIXED).propagate()
    assert rel_l2(got, c1_oracle()) < MIXED_TOL


def test_duct_small_fp64_parity():
    pb = duct_small()
    got = swkb.Plan(pb).propagate()
    assert rel_l2(got, duct_small_oracle()) < FP64_TOL


def test_duct_small_mixed_parity():
    pb = duct_small()
    got = swkb.Plan(pb, swkb.SWKB_MIXED).propagate()
    assert rel_l2(got, duct_small_oracle()) < MIXED_TOL


@pytest.mark.parametrize("bc", [w.BC_PERIODIC, w.BC_NEUMANN, w.BC_DIRICHLET])
@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, 1e-12), (swkb.SWKB_MIXED, 2e-5)])
def test_homogeneous_vs_angular_spectrum(bc, prec, tol):
    from refs import angular_spectrum
    pb = w.config_homogeneous(eps0=1.1, bc=bc, ray_stride=2, rk4_steps=3)
    got = swkb.Plan(pb, prec).propagate()
    g = geometry(pb)
    if bc == w.BC_PERIODIC:
        ref = angular_spectrum(pb.u0, pb.k, g.L, pb.dx * pb.n_screens, g.n_max, 1.1)
    else:
        sg = 1.0 if bc == w.BC_NEUMANN else -1.0
        n = pb.n_z
        full = np.zeros(2 * n, complex)
        full[n:] = pb.u0
        full[n - np.arange(1, n)] = sg * pb.u0[1:]
        ref = angular_spectrum(full, pb.k, g.L, pb.dx * pb.n_screens, g.n_max, 1.1)[n:]
    assert rel_l2(got, ref) < tol


def test_snapshots_and_resume_match_one_call():
    pb = w.config_unit_periodic()
    plan = swkb.Plan(pb)
    snaps = plan.propagate(snapshot_every=2)
    assert snaps.shape == (5, pb.n_z)
    whole = plan.propagate()
    assert np.array_equal(snaps[-1], whole)
    half = plan.propagate(n_screens=4)
    rest = plan.propagate(u0=half, q0=4, n_screens=6)
    assert np.array_equal(rest, whole)


def test_device_pointers_and_stream():
    torch = gpu()
    pb = w.config_unit_periodic(n_screens=3)
    s = torch.cuda.Stream()
    plan = swkb.Plan(pb, swkb.SWKB_MIXED, stream=s.cuda_stream)
    u0 = torch.from_numpy(pb.u0).cuda()
    out = torch.empty_like(u0)
    plan.propagate_device(u0.data_ptr(), out.data_ptr())
    host = plan.propagate()
    assert np.array_equal(out.cpu().numpy(), host)


def test_caustic_reported():
    pb = w.config_gaussian_medium(a=0.05, b=0.01, dx=100.0, n_screens=1)
    pr = pb.profile   # a taller table, so that the plan accepts the long screen
    pb = pb.with_(profile=w._table([0.0], -160.0, pr.dz, int(384 / pr.dz) + 1,
                                   [w.f_gaussian(0.05, 0.01, zc=32.0)]))
    with pytest.raises(swkb.SwkbError) as e:
        swkb.Plan(pb).propagate()
    assert e.value.status == swkb.SWKB_ERR_CAUSTIC


def test_turning_reported():
    k = 2 * math.pi
    prof = w._table([0.0, 20.0], -200.0, 0.125, 3201, [w.f_const(1.0), w.f_const(0.5)])
    z = 64.0 / 256 * np.arange(256)
    pb = w.Problem("turn", k, 0.0, 64.0, 256, w.BC_PERIODIC, 0.0, 20.0, 1, prof,
                   w.gaussian_beam(z, k, 32, 3, 0.0), math.radians(60.0), 1, 8)
    for prec in (swkb.SWKB_FP64, swkb.SWKB_MIXED):
        with pytest.raises(swkb.SwkbError) as e:
            swkb.Plan(pb, prec).propagate()
        assert e.value.status == swkb.SWKB_ERR_TURNING


def test_short_table_rejected_at_plan_creation():
    k = 2 * math.pi
    prof = w._table([0.0], -2.0, 0.125, 540, [w.f_const(1.0)])
    z = 64.0 / 256 * np.arange(256)
    pb = w.Problem("short", k, 0.0, 64.0, 256, w.BC_PERIODIC, 0.0, 20.0, 1, prof,
                   w.gaussian_beam(z, k, 32, 3, 0.0), math.radians(30.0), 1, 8)
    with pytest.raises(swkb.SwkbError) as e:
        swkb.Plan(pb)
    assert e.value.status == swkb.SWKB_ERR_INVALID_ARG


def test_full_size_duct_one_screen_fp64_vs_oracle():
    """Bench workload at full size (N_z = 16384, 977 modes): one screen from
    the antenna field through the same plan shape the benchmark times; the
    whole field is compared (the oracle finishes one screen in seconds)."""
    pb = w.config_surface_duct(n_screens=200)
    o = Oracle(pb)
    u = o.extend(pb.u0)
    want = o.screen(u, 7)
    got = swkb.Plan(pb).debug_screen(7, u)["u_next"]
    assert rel_l2(got, want) < FP64_TOL


def test_full_size_duct_mixed_vs_fp64_200_screens():
    """Whole 10 km / 200-screen bench workload: mixed path within 1e-4 of the
    FP64 path (the FP64 path is tied to the oracle above)."""
    pb = w.config_surface_duct()
    a = swkb.Plan(pb).propagate()
    b = swkb.Plan(pb, swkb.SWKB_MIXED).propagate()
    assert np.all(np.isfinite(a)) and np.linalg.norm(a) > 0.1 * np.linalg.norm(pb.u0)
    assert rel_l2(b, a) < MIXED_TOL


def test_paper_scale_one_screen_sampled_vs_oracle():
    """Paper-scale duct (N_z = 131072, 1395 modes, range-dependent profile
    with 101 columns): one screen mid-range through the same plan shape as
    the full 2000-screen run, compared with the oracle at sampled points."""
    pb = w.config_range_dependent_duct()
    o = Oracle(pb)
    u = o.extend(pb.u0)
    nz = pb.n_z
    dz = (pb.z_b - pb.z_a) / nz
    # across the 0.5 deg beam at 25 m, plus the ground and the upper air
    ms = [nz + int(round(z / dz)) for z in (23.1, 24.37, 25.0, 25.52, 26.9, 0.0, 140.0)]
    want = o.screen_points(u, 1000, ms)
    for prec, tol in ((swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)):
        got = swkb.Plan(pb, prec).propagate(q0=1000, n_screens=1)
        scale = np.max(np.abs(got))
        assert np.max(np.abs(got[np.array(ms) - nz] - want)) < tol * scale


def test_paper_scale_mixed_vs_fp64_first_screens():
    pb = w.config_range_dependent_duct()
    a = swkb.Plan(pb).propagate(n_screens=20)
    b = swkb.Plan(pb, swkb.SWKB_MIXED).propagate(n_screens=20)
    assert rel_l2(b, a) < MIXED_TOL


@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)])
def test_autotuned_plan_parity(prec, tol):
    """The autotuner only changes launch shapes: an autotuned plan still
    matches the oracle."""
    pb = duct_small()
    plan = swkb.Plan(pb, prec, autotune=True)
    assert plan.info.tile_points in (64, 128, 256, 512) and plan.info.fft_n1 >= 1
    assert rel_l2(plan.propagate(), duct_small_oracle()) < tol


@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)])
def test_fixed_launch_shapes(prec, tol):
    """Launch shapes an autotuned plan reports, given back as fixed shapes,
    rebuild the same plan without timing anything (bit-identical fields);
    other valid shapes still match the oracle; invalid ones are refused."""
    pb = duct_small()
    tuned = swkb.Plan(pb, prec, autotune=True)
    i = tuned.info
    shapes = (i.tile_points, i.ctas_per_sm, i.fft_n1)
    fixed = swkb.Plan(pb, prec, tiling=shapes)
    assert (fixed.info.tile_points, fixed.info.ctas_per_sm, fixed.info.fft_n1) == shapes
    assert fixed.info.mode_groups == i.mode_groups
    assert np.array_equal(fixed.propagate(), tuned.propagate())
    n = fixed.info.n_fft
    for sh in [(64, 1, 1), (128, 12, 2), (512, 3, min(64, n // 32))]:
        plan = swkb.Plan(pb, prec, tiling=sh)
        assert (plan.info.tile_points, plan.info.ctas_per_sm, plan.info.fft_n1) == sh
        assert rel_l2(plan.propagate(), duct_small_oracle()) < tol
    for bad in [(96, 4, 1), (1024, 4, 1), (128, 0, 1), (128, 4, 3), (128, 4, 128),
                (128, 4, 0), (0, 4, 2)]:
        with pytest.raises(swkb.SwkbError) as e:
            swkb.Plan(pb, prec, tiling=bad)
        assert e.value.status == swkb.SWKB_ERR_INVALID_ARG, bad


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_serial_timing(prec):
    """With serial timing the march runs on the plan's stream: same field, and
    the per-kernel event times of one propagation add up to no more than its
    wall time on the device."""
    torch = pytest.importorskip("torch")
    pb = duct_small()
    want = swkb.Plan(pb, prec).propagate()
    s = torch.cuda.Stream()
    plan = swkb.Plan(pb, prec, stream=s.cuda_stream)
    plan.set_timing(True, serial=True)
    u0 = torch.from_numpy(pb.u0).cuda()
    out = torch.empty_like(u0)
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    plan.propagate_device(u0.data_ptr(), out.data_ptr())   # graph capture
    plan.set_timing(True, serial=True)
    torch.cuda.synchronize()
    e0.record(s)
    plan.propagate_device(u0.data_ptr(), out.data_ptr())
    e1.record(s)
    torch.cuda.synchronize()
    st = plan.stats()
    assert np.array_equal(out.cpu().numpy(), want)
    assert st["kernel_timed"]["march"] == pb.n_screens
    total = sum(st["kernel_ms"].values())
    assert 0 < total <= e0.elapsed_time(e1) * 1.02 + 0.05
    plan.set_timing(False)


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_reuse_rays_identical_for_range_independent_media(prec):
    """The ray data depend only on the medium slab: with one table column,
    marching once per propagation gives bit-identical fields; with several
    columns the option is ignored."""
    pb = duct_small()
    a = swkb.Plan(pb, prec).propagate()
    plan = swkb.Plan(pb, prec, reuse_rays=True)
    plan.set_timing(True)
    b = plan.propagate()
    st = plan.stats()
    assert np.array_equal(a, b)
    assert st["kernel_launches"]["march"] == 1 and st["kernel_launches"]["resum"] == pb.n_screens
    c1 = w.config_unit_periodic(n_screens=6)
    assert np.array_equal(swkb.Plan(c1, prec, reuse_rays=True).propagate(),
                          swkb.Plan(c1, prec).propagate())


def test_fp32_medium_pieces():
    # FP32 plans evaluate the quintic table through cubic pieces: one per
    # interval where the profile is smooth on the table scale, 16 for the
    # duct (its 1 m blends set the curvature criterion), none in FP64
    duct = duct_small()
    assert swkb.Plan(duct, swkb.SWKB_MIXED).info.medium_pieces == 16
    assert swkb.Plan(duct, swkb.SWKB_FP64).info.medium_pieces == 0
    assert swkb.Plan(w.config_gaussian_medium(), swkb.SWKB_MIXED).info.medium_pieces == 1


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_rays_on_their_own_stream_give_identical_fields(prec, monkeypatch):
    # the overlapped sequence (march on a second stream, two ray-buffer sets)
    # runs the same kernels on the same arguments as the one-stream sequence:
    # snapshots and a range-dependent medium included, the fields are equal
    pb = duct_small()
    pr = pb.profile
    rd = pb.with_(profile=w._table([0.0, 150.0], pr.z0, pr.dz, pr.n_p,
                                   [w.f_trilinear_duct(12.0, -0.1), w.f_trilinear_duct(15.0, -0.1)]))
    for case in (pb, rd):
        monkeypatch.setenv("SWKB_OVERLAP", "0")
        one = swkb.Plan(case, prec).propagate(snapshot_every=2)
        monkeypatch.delenv("SWKB_OVERLAP")
        two = swkb.Plan(case, prec).propagate(snapshot_every=2)
        assert np.array_equal(one, two)


_batch_cache = {}


@pytest.mark.parametrize("idx", [12, 33], ids=["trilinear", "evaporation"])
@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)])
def test_uneven_batch_instances_match_oracle(idx, prec, tol):
    # two of the 64 uneven instances (seeded draw: frequency, height, N_z,
    # profile kind), the first two screens of each
    pb = w.batch_uneven(4, 64)[idx].with_(n_screens=2)
    if idx not in _batch_cache:
        _batch_cache[idx] = Oracle(pb).propagate(pb.u0)
    got = swkb.Plan(pb, prec).propagate()
    assert rel_l2(got, _batch_cache[idx]) < tol
