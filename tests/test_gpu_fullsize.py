"""Full-size parity: the GPU path against the FP64 CPU oracle on whole fields
of the benchmark-sized workloads, at both bars (FP64 rel-L2 <= 1e-9, mixed
rel-L2 <= 1e-4), with the oracle spread over the host's cores (bit-identical
to the serial oracle; tests/test_oracle_parallel.py).

  - surface duct, N_z = 16384 (977 modes, 2086 rays per mode): the first 10
    consecutive screens, every screen's field;
  - paper-scale range-dependent duct, N_z = 131072 (1395 modes, 101 table
    columns): one whole screen mid-range (screen 1000, 50 km);
  - the 64-instance uneven batch: the first screen of every instance.

The measured errors are printed (run with -s to see them)."""
import numpy as np
import pytest

from paper_2301_03814_gb300 import swkb
from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import rel_l2
from oracle.swkb_parallel import OraclePool, ParallelOracle

pytestmark = [pytest.mark.gpu, pytest.mark.slow]

FP64_TOL = 1e-9
MIXED_TOL = 1e-4
PRECS = [(swkb.SWKB_FP64, FP64_TOL), (swkb.SWKB_MIXED, MIXED_TOL)]
NAMES = {swkb.SWKB_FP64: "fp64", swkb.SWKB_MIXED: "mixed"}


@pytest.fixture(scope="module")
def pool():
    torch = pytest.importorskip("torch")
    if not torch.cuda.is_available():
        pytest.skip("no CUDA device")
    with OraclePool() as p:
        yield p


_want = {}


def _oracle(key, fn):
    if key not in _want:
        _want[key] = fn()
    return _want[key]


@pytest.mark.parametrize("prec,tol", PRECS, ids=["fp64", "mixed"])
def test_surface_duct_16384_ten_screens_whole_field(pool, prec, tol):
    pb = w.config_surface_duct().with_(n_screens=10)

    def run():
        with ParallelOracle(pb, pool=pool) as o:
            return np.array(o.propagate(pb.u0, snapshots=True)[1])
    want = _oracle("duct", run)
    got = swkb.Plan(pb, prec, autotune=True).propagate(snapshot_every=1)
    errs = [rel_l2(got[q], want[q]) for q in range(pb.n_screens)]
    print(f"\nPARITY surface-duct-16384 {NAMES[prec]} screens 1-10: max rel-L2 {max(errs):.3e}, "
          f"screen 10 {errs[-1]:.3e}")
    assert max(errs) < tol


@pytest.mark.parametrize("prec,tol", PRECS, ids=["fp64", "mixed"])
def test_paper_scale_duct_131072_one_whole_screen(pool, prec, tol):
    pb = w.config_range_dependent_duct()
    q = 1000

    def run():
        with ParallelOracle(pb, pool=pool) as o:
            return o.propagate(pb.u0, q0=q, n_screens=1)
    want = _oracle("paper", run)
    got = swkb.Plan(pb, prec, autotune=(prec == swkb.SWKB_MIXED)).propagate(q0=q, n_screens=1)
    err = rel_l2(got, want)
    print(f"\nPARITY range-dependent-duct-131072 {NAMES[prec]} screen {q}: rel-L2 {err:.3e}")
    assert err < tol


@pytest.mark.parametrize("prec,tol", PRECS, ids=["fp64", "mixed"])
def test_uneven_batch_first_screen_of_all_64(pool, prec, tol):
    batch = [pb.with_(n_screens=1) for pb in w.batch_uneven(4, 64)]

    def run():
        out = []
        for pb in batch:
            with ParallelOracle(pb, pool=pool) as o:
                out.append(o.propagate(pb.u0))
        return out
    want = _oracle("batch", run)
    errs = []
    for pb, ref in zip(batch, want):
        plan = swkb.Plan(pb, prec)
        errs.append(rel_l2(plan.propagate(), ref))
        plan.close()
    print(f"\nPARITY uneven-batch-64 {NAMES[prec]} first screen: max rel-L2 {max(errs):.3e} "
          f"(instance {int(np.argmax(errs))}), median {float(np.median(errs)):.3e}")
    assert max(errs) < tol
