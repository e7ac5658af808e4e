"""The benchmark's CPU-baseline plumbing on CPU: the spawned oracle pool computes the same rows
as one in-process oracle call."""
import collections

import numpy as np

import bench
import synthetic as S
from oracle import oracle as O

Workload = collections.namedtuple("Workload", "dims grid dirs T lo hi")


def test_oracle_pool_matches_serial():
    dims = [9, 7, 5]
    grid = S.uniform_u8_grid(dims, seed=11)
    dirs = S.fibonacci_directions(6)
    wl = Workload(dims, grid, dirs, 17, -1.8, 1.8)
    pool = bench.OraclePool(wl, 2)
    try:
        rows = pool.pool.map(bench._oracle_worker, range(len(dirs)), chunksize=1)
        assert pool.sample() > 0.0
    finally:
        pool.close()
    ref = O.wect_cubical(dims, grid.ravel().astype(np.int64), dirs, 17, -1.8, 1.8)
    assert np.array_equal(np.stack(rows), ref)
    assert bench.host_cores() >= 1
