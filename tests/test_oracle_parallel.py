"""The oracle's process-parallel local solves (the all-cores CPU baseline) give
the serial oracle's results bit for bit: same factors, same solves, only the
process that runs them differs."""
import numpy as np
import pytest

import workloads as W
from oracle import Decomposition, Sweeper
from oracle.parallel import PoolSweeper


@pytest.mark.parametrize("transmission", ["optimized", "habc"])
def test_pool_sweeper_equals_serial_sweeper(transmission):
    w = W.workload("custom", n=60, N1=3, N2=2, medium="layered", seed=3,
                   xcuts=[0, 21, 39, 60], ycuts=[0, 33, 60])
    args = (w.n, w.h, w.omega, w.m2, w.xcuts, w.ycuts)
    kw = dict(transmission=transmission)
    serial = Sweeper(Decomposition(*args, **kw))
    pool = PoolSweeper(Decomposition(*args, **kw), args, kw, processes=2)
    try:
        r = W.random_complex((1, w.N), 5)[0]
        for kind in ("BSP", "SP"):
            assert np.array_equal(pool.precondition(r, kind), serial.precondition(r, kind)), kind
        x = serial.dec.unflatten(W.random_complex((1, serial.dec.flatten(serial.dec.zero_trace()).size), 6)[0])
        assert all(np.array_equal(a, b) for a, b in zip(pool.apply_S(x).values(), serial.apply_S(x).values()))
    finally:
        pool.close()
