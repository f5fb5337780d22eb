"""The bench's multi-core evaluation of the oracle (cpu_baseline and --impl reference legs), on the CPU.

It splits the oracle's element loop over a process pool; its F(u) and J(u)^T v must equal the
oracle's own Grid.rhs and Grid.jacT up to the grouping of the gather-scatter sums."""
import numpy as np
import pytest

import bench
from oracle.sem import Grid


@pytest.mark.parametrize("dim,E,N,procs", [(3, 4, 3, 3), (3, 3, 4, 2), (2, 6, 5, 4), (2, 5, 3, 1), (1, 8, 7, 3)])
def test_pooled_operators_equal_the_oracle(dim, E, N, procs):
    g = Grid(dim, E, N, 0.02)
    rng = np.random.default_rng(dim * 100 + E * 10 + N)
    u = rng.standard_normal((dim,) + g.global_shape())
    v = rng.standard_normal((dim,) + g.global_shape())
    pool = bench.OraclePool(g, procs)
    try:
        F, JT = pool.rhs(u), pool.jacT(u, v)
        F2 = pool.rhs(v)           # the shared buffers carry no state between calls
    finally:
        pool.close()
    for got, ref in ((F, g.rhs(u)), (JT, g.jacT(u, v)), (F2, g.rhs(v))):
        assert np.max(np.abs(got - ref)) <= 1e-13 * np.max(np.abs(ref))
