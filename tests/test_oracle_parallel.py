"""The oracle spread over host processes gives the serial oracle's fields bit
for bit (same arithmetic, terms added in mode order) and fails where it fails
(which R7 event is met first may differ when different modes meet different
ones: each worker checks its own slice of modes)."""
import numpy as np
import pytest

from paper_2301_03814_gb300 import workloads as w
from oracle.swkb_oracle import Oracle, OracleError
from oracle.swkb_parallel import ParallelOracle


@pytest.mark.parametrize("make", [lambda: w.config_unit_periodic(n_screens=3),
                                  lambda: w.config_surface_duct_small(n_screens=2)],
                         ids=["periodic-two-columns", "grounded-duct"])
def test_parallel_oracle_is_bit_identical_to_serial(make):
    pb = make()
    want, wsnaps = Oracle(pb).propagate(pb.u0, snapshots=True)
    with ParallelOracle(pb, workers=3) as po:
        got, gsnaps = po.propagate(pb.u0, snapshots=True)
        assert np.array_equal(got, want)
        assert all(np.array_equal(a, b) for a, b in zip(gsnaps, wsnaps))
        # resume from a snapshot at screen 1
        tail = po.propagate(gsnaps[0], q0=1, n_screens=pb.n_screens - 1)
        assert np.array_equal(tail, want)


def test_parallel_oracle_raises_the_serial_errors():
    pb = w.config_gaussian_medium(a=0.05, b=0.01, dx=100.0, n_screens=1)
    with pytest.raises(OracleError):
        Oracle(pb).propagate(pb.u0)
    with ParallelOracle(pb, workers=2) as po:
        with pytest.raises(OracleError):
            po.propagate(pb.u0)


def test_one_pool_serves_several_problems():
    from oracle.swkb_parallel import OraclePool
    pbs = [w.config_unit_periodic(n_screens=1), w.config_surface_duct_small(n_screens=1)]
    with OraclePool(2) as pool:
        for pb in pbs + pbs[:1]:
            with ParallelOracle(pb, pool=pool) as po:
                assert np.array_equal(po.propagate(pb.u0), Oracle(pb).propagate(pb.u0))
