"""The batching workload's seeded family: deterministic, uneven, alias-free grids."""

import numpy as np

import synth


def test_batch_family_sizes_and_determinism():
    a = synth.batch_family(16, seed=0)
    b = synth.batch_family(16, seed=0)
    assert a == b
    grids = sorted({sp.grid[0] for sp in a})
    assert grids[0] == 32 and grids[-1] == 80 and len(grids) >= 10
    for sp in a:
        n = sp.grid[0]
        m = n
        for p in (2, 3, 5):
            while m % p == 0:
                m //= p
        assert m == 1  # 2,3,5-smooth
        assert sp.nocc == 2 * sp.natom and 8 <= sp.nocc <= 160
        s = synth.make_system(sp) if n <= 40 else None
        if s is not None:
            # alias-free: the product of two sphere functions fits the grid
            nmax = np.abs(s.miller).max()
            assert n >= 3 * nmax + 1
