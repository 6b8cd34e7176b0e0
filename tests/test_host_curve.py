"""The library's coercive field (mm_coercive_field, host code of the C-ABI:
no GPU needed) against the oracle's definition (oracle/curve.py, Sec. 3.1:
the applied field where M along the sweep changes sign, linearly
interpolated), on hand-made and random curves and the edge cases."""
import os

import numpy as np
import pytest

from oracle import curve


@pytest.fixture(scope="module")
def hc():
    from paper_1801_03690_gb300 import _lib, coercive_field, MMError
    if not os.path.exists(_lib.LIB_PATH):
        pytest.skip("library not built (run __graft_entry__.build())")
    return coercive_field, MMError


def test_hand_made_curve(hc):
    fields = np.array([[0, 0, 0.0], [0, 0, -1.0], [0, 0, -2.0], [0, 0, -3.0]])
    M = np.array([[0, 0, 1.0], [0, 0, 0.5], [0, 0, -0.5], [0, 0, -1.0]])
    assert hc[0](fields, M) == pytest.approx(1.5, abs=1e-15)
    assert hc[0](fields, np.abs(M)) is None


def test_random_curves_match_oracle(hc):
    rng = np.random.default_rng(7)
    for trial in range(200):
        n = int(rng.integers(2, 40))
        d = rng.standard_normal(3)
        d /= np.linalg.norm(d)
        b = np.linspace(rng.uniform(-1, 1), rng.uniform(-9, -1), n)
        fields = b[:, None] * d[None, :] + 1e-3 * rng.standard_normal((n, 3))
        s = np.cumsum(rng.uniform(-0.3, 0.1, n)) + rng.uniform(0, 2)
        M = s[:, None] * d[None, :] + 0.05 * rng.standard_normal((n, 3))
        ref = curve.coercive_field(fields, M)
        got = hc[0](fields, M)
        if ref is None:
            assert got is None, trial
        else:
            assert got == pytest.approx(ref, rel=1e-14, abs=1e-15), trial


def test_exact_zero_and_equal_ends(hc):
    fields = np.array([[0, 0, 0.0], [0, 0, -1.0], [0, 0, -2.0]])
    M = np.array([[0, 0, 1.0], [0, 0, 0.0], [0, 0, -1.0]])
    assert hc[0](fields, M) == pytest.approx(curve.coercive_field(fields, M))
    loop = np.array([[0, 0, 1.0], [0, 0, -1.0], [0, 0, 1.0]])      # ends coincide: u = last field
    Ml = np.array([[0, 0, 1.0], [0, 0, -1.0], [0, 0, 1.0]])
    assert hc[0](loop, Ml) == pytest.approx(curve.coercive_field(loop, Ml))


def test_rejects_bad_input(hc):
    coercive_field, MMError = hc
    with pytest.raises(MMError):
        coercive_field(np.zeros((1, 3)), np.ones((1, 3)))
    with pytest.raises(MMError):
        coercive_field(np.zeros((3, 3)), np.ones((3, 3)))             # zero sweep direction
    with pytest.raises(MMError):
        coercive_field(np.array([[0, 0, 0.0], [0, 0, np.nan]]), np.ones((2, 3)))
