"""Failure detection on the device without a fault: every device-side wait of the
library is bounded and turns into SBFWI_ETIMEOUT, after which the context is still
usable.  The wait is made to run out by blocks that never arrive at the barrier."""

import numpy as np
import pytest

from sbfwi_inputs import tiny_workload

pytestmark = pytest.mark.gpu


def test_barrier_completes_when_every_block_arrives(lib):
    assert lib.selftest_barrier(8, 0, rounds=50) == lib.OK
    assert lib.selftest_barrier(152, 0, rounds=20) == lib.OK


@pytest.mark.parametrize("n_blocks,n_absent", [(2, 1), (8, 3), (152, 1)])
def test_barrier_times_out_when_a_block_never_arrives(lib, n_blocks, n_absent):
    assert lib.selftest_barrier(n_blocks, n_absent, budget_cycles=2_000_000) == lib.ETIMEOUT


def test_device_is_usable_after_a_timeout(lib):
    w = tiny_workload(K=40)
    M = lib.Mesh.from_inputs(w.mesh, w.n_r)
    md = lib.Model(M, w.c, w.rho_true, w.dt)
    before, _ = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    assert lib.selftest_barrier(4, 1, budget_cycles=1_000_000) == lib.ETIMEOUT
    after, _ = lib.forward(md, w.src_nodes, w.wavelets, w.rec_nodes, keep=False)
    assert np.array_equal(before, after)
    assert lib.selftest_barrier(4, 0) == lib.OK


def test_selftest_rejects_bad_arguments(lib):
    for args in [(0, 0), (4, 4), (4, -1)]:
        with pytest.raises(lib.SbfwiError) as ei:
            lib.selftest_barrier(*args)
        assert ei.value.code == lib.EINVAL
    with pytest.raises(lib.SbfwiError):
        lib.selftest_barrier(4, 1, budget_cycles=10)
    with pytest.raises(lib.SbfwiError):
        lib.selftest_barrier(1_000_000, 0)
