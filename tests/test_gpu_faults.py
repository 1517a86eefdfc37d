"""Failures injected on the host (no GPU fault): a plan whose n-th device
allocation is refused (SWKB_FAIL_ALLOC_AT) fails cleanly with SWKB_ERR_OOM,
releases what it had allocated, and leaves the library usable; the request
server reports the same failure through swkb_poll and serves the next
request."""
import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def torch():
    t = pytest.importorskip("torch")
    if not t.cuda.is_available():
        pytest.skip("no CUDA device")
    return t


@pytest.mark.parametrize("prec", [swkb.SWKB_FP64, swkb.SWKB_MIXED])
def test_refused_allocations_fail_cleanly(torch, monkeypatch, prec):
    pb = w.config_unit_periodic(n_screens=2)
    want = swkb.Plan(pb, prec).propagate()
    torch.cuda.synchronize()
    free0 = torch.cuda.mem_get_info()[0]
    refused = 0
    for n in range(1, 64):
        monkeypatch.setenv("SWKB_FAIL_ALLOC_AT", str(n))
        try:
            plan = swkb.Plan(pb, prec)
        except swkb.SwkbError as e:
            assert e.status == swkb.SWKB_ERR_OOM
            refused += 1
            continue
        plan.close()          # n is past the plan's last allocation
        break
    monkeypatch.delenv("SWKB_FAIL_ALLOC_AT")
    assert refused >= 10      # every allocation point of plan creation was exercised
    torch.cuda.synchronize()
    assert abs(torch.cuda.mem_get_info()[0] - free0) < (32 << 20)   # nothing leaked
    assert np.array_equal(swkb.Plan(pb, prec).propagate(), want)


def test_server_reports_a_refused_allocation_and_serves_the_next_request(torch, monkeypatch):
    pb = w.config_unit_periodic(n_screens=2)
    want = swkb.Plan(pb, swkb.SWKB_MIXED).propagate()
    srv = swkb.Server(8 << 30, max_slots=2)
    try:
        monkeypatch.setenv("SWKB_FAIL_ALLOC_AT", "3")
        st, t = srv.submit(pb, swkb.SWKB_MIXED)
        assert st == swkb.SWKB_OK
        st, _ = srv.poll(t, timeout_ms=-1)
        assert st == swkb.SWKB_ERR_OOM
        monkeypatch.delenv("SWKB_FAIL_ALLOC_AT")
        st, t = srv.submit(pb, swkb.SWKB_MIXED)
        assert st == swkb.SWKB_OK
        st, out = srv.poll(t, timeout_ms=-1)
        assert st == swkb.SWKB_OK
        assert np.array_equal(np.asarray(out).reshape(-1), want)
    finally:
        srv.close()
