"""The oracle's OpenMP build, used only to time the oracle on every host
core, computes the same states as its one-thread build: rows, wavenumbers and
nodes are independent in the method (Sec. IV.2 collision per node, streaming
per population and node, Sec. IV.3 transforms per row and solves per
wavenumber), so sharing them among threads changes no arithmetic.  Only the
diagnostic sums are reordered."""
import numpy as np
import pytest

import oracle as o
import workloads as wl


def test_openmp_build_gives_bitwise_the_same_state():
    w = wl.Workload("threads", 64, 52, 190.0, amp=[1e-3, 5e-4], phase=[0.4, 1.3])
    p = o.setup(*w.args())
    s1 = o.init_state(p, w.amp, w.phase)
    d1 = o.step(s1, 30, diag=True)
    n = o.use_threads(4)
    try:
        if n == 0:
            pytest.skip("no OpenMP build of the oracle on this host")
        p2 = o.setup(*w.args())
        s2 = o.init_state(p2, w.amp, w.phase)
        d2 = o.step(s2, 30, diag=True)
    finally:
        o.use_one_thread()
    assert np.array_equal(s1.f, s2.f) and np.array_equal(s1.g, s2.g) and np.array_equal(s1.phi, s2.phi)
    np.testing.assert_allclose(d2, d1, rtol=1e-12, atol=1e-15)
