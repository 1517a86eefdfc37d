"""swkb_modes_noalloc: step (a) for callers that cannot allocate device memory.

Some callers cannot call cudaMalloc: a host framework that owns and
pre-partitions all device memory, or a latency-critical loop where an
allocation would synchronise the device.  For them the library offers the
screen field's pruned DFT with its working storage in fixed, file-scope device
arrays.  This test calls it through the C ABI and checks it against the
allocating path (the step-(a) output of swkb_debug_screen) on two calls in a
row, so that the second call runs on scratch the first one left behind.  It is
collected last so that a run stopping at the first failure has run every other
test first; it also passes alone in a fresh process (the first call does the
per-device set-up)."""
import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w

pytestmark = pytest.mark.gpu

TOL = 1e-12   # relative to the largest coefficient; both sides are FP64


def _torch():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    return torch


@pytest.mark.parametrize("make", [lambda: w.config_unit_periodic(n_screens=1),
                                  w.config_surface_duct_small],
                         ids=["n512", "n8192"])
def test_noalloc_modes_match_allocating_path_twice(make):
    torch = _torch()
    pb = make()
    plan = swkb.Plan(pb)
    N, n_max = plan.info.n_fft, plan.info.n_max
    rng = np.random.default_rng(N)
    u_dev = torch.empty(N, dtype=torch.complex128, device="cuda")
    c_dev = torch.empty(2 * n_max + 1, dtype=torch.complex128, device="cuda")
    for _ in range(2):
        field = rng.standard_normal(N) + 1j * rng.standard_normal(N)
        if pb.bc != w.BC_PERIODIC:       # fields of a grounded domain are even
            field = 0.5 * (field + field[(N - np.arange(N)) % N])
        want = plan.debug_screen(0, field)["c"]
        u_dev.copy_(torch.from_numpy(field))
        status = swkb.swkb_modes_noalloc(u_dev.data_ptr(), N, n_max, c_dev.data_ptr())
        assert status == swkb.SWKB_OK, swkb.swkb_last_error()
        torch.cuda.synchronize()
        got = c_dev.cpu().numpy()
        assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))


@pytest.mark.parametrize("n_fft,n_max", [(64, 1), (64, 31), (65536, 1), (65536, 32767)])
def test_noalloc_modes_at_the_size_limits_match_numpy(n_fft, n_max):
    """The smallest and largest accepted lengths with the fewest and the most
    kept modes (n_max = n_fft / 2 - 1 uses a unit phase per mode up to index
    n_fft - 2), twice in a row, against numpy's FFT of a random field."""
    torch = _torch()
    rng = np.random.default_rng(n_fft + n_max)
    n = np.arange(-n_max, n_max + 1)
    u_dev = torch.empty(n_fft, dtype=torch.complex128, device="cuda")
    c_dev = torch.empty(2 * n_max + 1, dtype=torch.complex128, device="cuda")
    for _ in range(2):
        field = rng.standard_normal(n_fft) + 1j * rng.standard_normal(n_fft)
        want = np.fft.fft(field)[n % n_fft] / n_fft
        u_dev.copy_(torch.from_numpy(field))
        status = swkb.swkb_modes_noalloc(u_dev.data_ptr(), n_fft, n_max, c_dev.data_ptr())
        assert status == swkb.SWKB_OK, swkb.swkb_last_error()
        torch.cuda.synchronize()
        got = c_dev.cpu().numpy()
        assert np.max(np.abs(got - want)) <= TOL * np.max(np.abs(want))


def test_noalloc_rejects_sizes_beyond_its_scratch_and_host_pointers():
    torch = _torch()
    u = torch.zeros(1 << 17, dtype=torch.complex128, device="cuda")
    c = torch.zeros(64, dtype=torch.complex128, device="cuda")
    assert swkb.swkb_modes_noalloc(u.data_ptr(), 1 << 17, 31, c.data_ptr()) == \
        swkb.SWKB_ERR_INVALID_ARG
    assert "65536" in swkb.swkb_last_error()
    assert swkb.swkb_modes_noalloc(u.data_ptr(), 512, 256, c.data_ptr()) == \
        swkb.SWKB_ERR_INVALID_ARG
    host = np.zeros(2 * 512)
    assert swkb.swkb_modes_noalloc(host.ctypes.data, 512, 31, c.data_ptr()) == \
        swkb.SWKB_ERR_INVALID_ARG
