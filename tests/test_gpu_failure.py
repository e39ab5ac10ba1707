"""Failure handling on the GPU without a fault: a bounded device-side wait runs out.

Every mbarrier wait of the tensor-core kernels gives up after a cycle limit and records a
time-out in the handle's sticky flags.  afqmc_kp_wait_selftest runs that wait on a barrier
that nothing arrives at (a few thousand cycles), with nothing in flight; the test expects the
time-out status from afqmc_kp_last_error and a device that still computes correct results.
"""
import numpy as np
import pytest

import gen

torch = pytest.importorskip("torch")
from gpu_util import dev, host, make, oracle_energy  # noqa: E402

pytestmark = pytest.mark.gpu

TIMEOUT = 5


@pytest.mark.parametrize("precision", ["mixed", "fp64"])
def test_bounded_wait_times_out_and_the_device_still_answers(precision):
    spec = gen.SystemSpec(grid=(1, 1, 2), M=6, nocc=2, nchol=5, nwalkers=3, random_trial=True, seed=4)
    sys_, osys = make(spec, precision)
    assert sys_.last_error() == (0, 0)
    # the arrival comes first: the wait returns at once, no flag
    sys_.wait_selftest(arrive=True, limit_cycles=4000)
    assert sys_.last_error() == (0, 0)
    # nothing arrives: the wait gives up after 4000 cycles and records a time-out
    sys_.wait_selftest(arrive=False, limit_cycles=4000)
    assert sys_.last_error() == (TIMEOUT, 0)
    assert sys_.last_error() == (0, 0)          # read and cleared
    # the context is intact: the next call computes the right energies
    phis = gen.near_trial_walkers(spec)
    e = host(sys_.local_energy(dev(phis)))
    ref = oracle_energy(osys, phis)
    assert np.abs(e - ref).max() / spec.nk < 1e-5
    assert sys_.last_error() == (0, 0)
    sys_.close()


def test_wait_selftest_rejects_limits_out_of_range():
    from paper_2003_09468_gb300 import AfqmcError
    spec = gen.SystemSpec(grid=(1, 1, 1), M=4, nocc=1, nchol=2, nwalkers=1)
    sys_, _ = make(spec, "fp64")
    for bad in (0, -5, (1 << 31) + 1):
        with pytest.raises(AfqmcError):
            sys_.wait_selftest(arrive=False, limit_cycles=bad)
    assert sys_.last_error() == (0, 0)
    sys_.close()
