"""L-BFGS (Table I's optimiser): the library's host implementation and the
oracle's, pinned to closed-form minimisers (no GPU: host arithmetic)."""
import numpy as np
import pytest

import oracle
from paper_2404_12134_gb300 import _abi, build


@pytest.fixture(scope="module")
def api():
    build.build()
    _abi.load()
    from paper_2404_12134_gb300 import api as a
    return a


def _quadratic(n=20, seed=70):
    rng = np.random.default_rng(seed)
    Q, _ = np.linalg.qr(rng.normal(size=(n, n)))
    A = Q @ np.diag(np.linspace(1.0, 100.0, n)) @ Q.T
    b = rng.normal(size=n)

    def fn(x):
        return 0.5 * x @ A @ x - b @ x, A @ x - b
    return fn, np.linalg.solve(A, b)


def _rosenbrock(x):
    f = 100.0 * (x[1] - x[0] ** 2) ** 2 + (1 - x[0]) ** 2
    g = np.array([-400.0 * x[0] * (x[1] - x[0] ** 2) - 2 * (1 - x[0]), 200.0 * (x[1] - x[0] ** 2)])
    return f, g


def test_quadratic_minimiser(api):
    """An SPD quadratic (condition 100): both implementations reach A^-1 b
    (numpy's solve) to 1e-6, stopping on the gradient tolerance."""
    fn, xs = _quadratic()
    x0 = np.zeros_like(xs)
    for impl in ("lib", "oracle"):
        if impl == "lib":
            x, f, it, ev, why = api.lbfgs_minimize(fn, x0, api.lbfgs_params(max_iter=500, max_fun=2000, gtol=1e-9, ftol=0.0))
        else:
            x, f, it, ev, why = oracle.lbfgs(fn, x0, max_iter=500, max_fun=2000, gtol=1e-9, ftol=0.0)
        assert why in ("gtol", "ftol"), impl      # at machine precision f stops decreasing (rel = 0 <= ftol)
        assert np.max(np.abs(x - xs)) <= 1e-6, impl


def test_rosenbrock(api):
    x0 = np.array([-1.2, 1.0])
    for impl in ("lib", "oracle"):
        if impl == "lib":
            x, f, it, ev, why = api.lbfgs_minimize(_rosenbrock, x0, api.lbfgs_params(max_iter=500, max_fun=5000, ftol=0.0))
        else:
            x, f, it, ev, why = oracle.lbfgs(_rosenbrock, x0, max_iter=500, max_fun=5000, ftol=0.0)
        assert np.max(np.abs(x - 1.0)) <= 1e-5 and f <= 1e-10, impl


def test_library_follows_the_oracle(api):
    """The same method step by step: iteration and evaluation counts equal
    and the iterates equal to rounding on the quadratic and Rosenbrock."""
    fn, xs = _quadratic(12, 71)
    for f_, x0 in ((fn, np.ones(12)), (_rosenbrock, np.array([-1.2, 1.0]))):
        a = api.lbfgs_minimize(f_, x0, api.lbfgs_params(max_iter=30, max_fun=300))
        b = oracle.lbfgs(f_, x0, max_iter=30, max_fun=300)
        assert a[2:] == b[2:]
        assert np.allclose(a[0], b[0], rtol=1e-9, atol=1e-12)


def test_stopping_rules(api):
    fn, xs = _quadratic()
    x0 = np.zeros_like(xs)
    x, f, it, ev, why = api.lbfgs_minimize(fn, x0, api.lbfgs_params(max_iter=3))
    assert why == "max_iter" and it == 3
    x, f, it, ev, why = api.lbfgs_minimize(fn, x0, api.lbfgs_params(max_fun=4, ftol=0.0))
    assert why == "max_fun" and ev <= 4
    # relative reduction below ftol: a flat objective stops after one step
    x, f, it, ev, why = api.lbfgs_minimize(lambda x: (1e-9 * float(x @ x), 2e-9 * x), np.ones(3))
    assert why in ("ftol", "gtol") and it <= 1
