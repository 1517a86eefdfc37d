"""Batched propagation in one persistent launch (swkb_batch_*): every
request's field equals its own plan's field bit for bit (same kernels'
arithmetic, launch shapes and summation orders), the batch matches the oracle
at both bars, reruns and new inputs work, and a wait that cannot be satisfied
runs out into SWKB_ERR_TIMEOUT with the device still usable."""
import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import rel_l2

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module", autouse=True)
def _need_gpu():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")


def uneven():
    """Periodic and grounded problems of different sizes and screen counts
    (1 to 7 screens: the three ray-buffer sets rotate), one range-dependent
    medium (two table columns), two uneven-batch instances."""
    c4 = w.batch_uneven(4, 64)
    return [
        w.config_unit_periodic(n_screens=7),
        w.config_surface_duct_small(n_screens=5),
        w.config_unit_periodic(n_screens=1),
        w.config_surface_duct_small(n_screens=2, n_z=2048, height=25.0),
        w.config_homogeneous(bc=w.BC_DIRICHLET, ray_stride=2),
        c4[12].with_(n_screens=4),
        c4[33].with_(n_screens=3),
    ]


@pytest.mark.parametrize("prec", [swkb.SWKB_MIXED, swkb.SWKB_FP64], ids=["mixed", "fp64"])
def test_batch_fields_equal_plans_alone_bit_for_bit(prec):
    pbs = uneven()
    alone = [swkb.Plan(pb, prec).propagate() for pb in pbs]
    b = swkb.Batch(pbs, prec)
    assert b.info.instances == len(pbs) and b.info.grid >= 152
    got = b.run()
    for i, (g, a) in enumerate(zip(got, alone)):
        assert np.array_equal(g, a), (i, rel_l2(g, a))
    # a second run replays the captured launch and gives the same fields
    again = b.run()
    assert all(np.array_equal(g, a) for g, a in zip(again, alone))
    b.close()


_oracle = {}


@pytest.mark.parametrize("prec,tol", [(swkb.SWKB_FP64, 1e-9), (swkb.SWKB_MIXED, 1e-4)],
                         ids=["fp64", "mixed"])
def test_batch_of_uneven_instances_matches_oracle(prec, tol):
    from oracle.swkb_parallel import OraclePool, ParallelOracle
    c4 = w.batch_uneven(4, 64)
    pbs = [c4[i].with_(n_screens=2) for i in (0, 12, 33, 50)]
    got = swkb.Batch(pbs, prec).run()
    if "want" not in _oracle:
        with OraclePool() as pool:
            want = []
            for pb in pbs:
                with ParallelOracle(pb, pool=pool) as o:
                    want.append(o.propagate(pb.u0))
        _oracle["want"] = want
    for g, ref in zip(got, _oracle["want"]):
        assert rel_l2(g, ref) < tol


def test_batch_new_inputs_and_device_buffers():
    torch = pytest.importorskip("torch")
    pbs = uneven()[:4]
    b = swkb.Batch(pbs, swkb.SWKB_MIXED)
    rng = np.random.default_rng(7)
    fields = []
    for pb in pbs:
        f = pb.u0 * (1.0 + 0.2 * rng.standard_normal(pb.n_z))
        if pb.bc != w.BC_PERIODIC:
            f[0] = pb.u0[0]
        fields.append(f.astype(np.complex128))
    want = [swkb.Plan(pb, swkb.SWKB_MIXED).propagate(u0=f) for pb, f in zip(pbs, fields)]
    got = b.run(fields)
    assert all(np.array_equal(g, a) for g, a in zip(got, want))
    din = torch.from_numpy(np.concatenate(fields)).cuda()
    dout = torch.empty_like(din)
    b.run_device(din.data_ptr(), dout.data_ptr())
    host = dout.cpu().numpy()
    for i, a in enumerate(want):
        assert np.array_equal(host[b.offsets[i]:b.offsets[i + 1]], a)
    b.close()


def test_full_uneven_batch_three_screens_equals_plans_alone():
    pbs = [pb.with_(n_screens=3) for pb in w.batch_uneven(4, 64)]
    b = swkb.Batch(pbs, swkb.SWKB_MIXED)
    got = b.run()
    b.close()
    for i in range(0, 64, 7):
        assert np.array_equal(got[i], swkb.Plan(pbs[i], swkb.SWKB_MIXED).propagate()), i


def test_batch_rejects_bad_requests():
    pbs = uneven()[:2]
    with pytest.raises(swkb.SwkbError) as e:
        swkb.Batch([pbs[0], pbs[1].with_(n_screens=0)], swkb.SWKB_MIXED)
    assert e.value.status == swkb.SWKB_ERR_INVALID_ARG


def test_unsatisfiable_wait_runs_out(monkeypatch):
    """A test hook gives one work item a producer that never finishes: its
    bounded wait runs out, every CTA leaves, the run returns
    SWKB_ERR_TIMEOUT, and the device keeps working."""
    pbs = uneven()[:3]
    monkeypatch.setenv("SWKB_BATCH_STALL", "1")
    b = swkb.Batch(pbs, swkb.SWKB_MIXED, wait_limit_ms=50)
    monkeypatch.delenv("SWKB_BATCH_STALL")
    assert b.run_status() == swkb.SWKB_ERR_TIMEOUT
    assert "wait limit" in swkb.swkb_last_error()
    assert b.run_status() == swkb.SWKB_ERR_TIMEOUT      # again, on the same batch
    b.close()
    ok = swkb.Batch(pbs, swkb.SWKB_MIXED).run()
    assert all(np.array_equal(g, swkb.Plan(pb, swkb.SWKB_MIXED).propagate())
               for g, pb in zip(ok, pbs))
