"""Host logic of the batched form: splitting the persistent grid into
per-problem teams (mm_batch_plan; no GPU needed)."""
import os

import numpy as np
import pytest

from paper_1801_03690_gb300 import _lib

pytestmark = pytest.mark.skipif(not os.path.exists(_lib.LIB_PATH), reason="library not built")


def plan(work, total, gamma=1.0):
    from paper_1801_03690_gb300 import batch_plan
    return batch_plan(work, total, gamma)


def test_plan_sums_and_minimum_one_block():
    rng = np.random.default_rng(0)
    for _ in range(50):
        n = int(rng.integers(1, 64))
        work = rng.integers(1, 10**7, size=n)
        total = int(rng.integers(n, 4 * 152 + 1))
        for g in (0.0, 0.5, 1.0, 1.5):
            b = plan(work, total, g)
            assert b.sum() == total
            assert b.min() >= 1


def test_plan_proportional_to_work():
    b = plan([100, 300, 600], 100, 1.0)
    assert list(b) == [10, 30, 60]
    b = plan([1, 1, 1, 1], 10, 1.0)
    assert sorted(b) == [2, 2, 3, 3] and b.sum() == 10
    b = plan([4, 16], 6, 0.5)        # sqrt: 2 : 4
    assert list(b) == [2, 4]
    b = plan([1, 10**9], 4, 1.0)     # tiny member still gets one block
    assert list(b) == [1, 3]


def test_plan_deterministic_and_rejects_bad_input():
    w = [5, 7, 11, 13]
    assert list(plan(w, 40)) == list(plan(w, 40))
    from paper_1801_03690_gb300 import MMError
    with pytest.raises(MMError):
        plan([1, 2, 3], 2)               # fewer blocks than members
    with pytest.raises(MMError):
        plan([1, -2], 10)
