"""Pins of Algorithm 1 (preconditioned linear CG) against dense linear
algebra."""
import numpy as np

from oracle.linear_cg import alg1


def _spd(n, seed, cond=1e3):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    ev = np.geomspace(1.0, cond, n)
    return (Q * ev) @ Q.T


def test_matches_dense_solve():
    C = _spd(40, 0)
    rng = np.random.default_rng(1)
    b = rng.normal(size=40)
    dinv = 1.0 / np.diag(C)
    x, steps, why = alg1(lambda v: C @ v, b, np.zeros(40), lambda g: dinv * g,
                         1e-12 * np.linalg.norm(b), 1000)
    assert why == "tol"
    np.testing.assert_allclose(x, np.linalg.solve(C, -b), rtol=1e-8, atol=1e-10)


def test_finite_termination_in_n_steps():
    C = _spd(12, 2, cond=10.0)
    b = np.arange(12.0) - 5
    x, steps, why = alg1(lambda v: C @ v, b, np.ones(12), lambda g: g.copy(),
                         1e-10 * np.linalg.norm(b), 1000)
    assert steps <= 12
    np.testing.assert_allclose(C @ x, -b, atol=1e-9)


def test_energy_norm_error_decreases():
    C = _spd(30, 3)
    b = np.random.default_rng(4).normal(size=30)
    xs = np.linalg.solve(C, -b)
    errs = []
    for k in range(1, 15):
        x, _, _ = alg1(lambda v: C @ v, b, np.zeros(30), lambda g: g.copy(), 0.0, k)
        e = x - xs
        errs.append(e @ C @ e)
    assert all(errs[i + 1] <= errs[i] * (1 + 1e-12) for i in range(len(errs) - 1))


def test_negative_curvature_exit():
    C = np.diag([1.0, -2.0, 3.0])
    b = np.array([0.0, 1.0, 0.0])
    x, steps, why = alg1(lambda v: C @ v, b, np.zeros(3), lambda g: g.copy(), 1e-12, 10,
                         neg_curvature=True)
    assert why == "neg_curvature" and steps == 1
    np.testing.assert_array_equal(x, 0.0)


def test_max_iter_exit():
    C = _spd(20, 5)
    b = np.ones(20)
    x, steps, why = alg1(lambda v: C @ v, b, np.zeros(20), lambda g: g.copy(), 0.0, 3)
    assert why == "max_iter" and steps == 3
