"""The BFGS minimiser and Hessian errors on functions with known minima (CPU)."""
import numpy as np

from paper_1702_06735_gb300 import minimize


def rosenbrock(x):
    f = sum(100.0 * (x[1:] - x[:-1] ** 2) ** 2 + (1 - x[:-1]) ** 2)
    g = np.zeros_like(x)
    g[:-1] = -400 * x[:-1] * (x[1:] - x[:-1] ** 2) - 2 * (1 - x[:-1])
    g[1:] += 200 * (x[1:] - x[:-1] ** 2)
    return float(f), g


def test_bfgs_rosenbrock():
    r = minimize.bfgs(rosenbrock, np.array([-1.2, 1.0, -0.5, 0.8]), gtol=1e-8, edm_tol=1e-16, max_iter=1000)
    assert r.converged
    assert np.allclose(r.x, 1.0, atol=1e-5)


def test_bfgs_respects_fixed_parameters_and_scales():
    A = np.diag([4.0, 1.0, 9.0])
    c = np.array([1.0, -2.0, 3.0])

    def quad(x):
        d = x - c
        return float(0.5 * d @ A @ d), A @ d
    r = minimize.bfgs(quad, np.zeros(3), floating=[True, False, True], scale=[1e-3, 1, 10.0], gtol=1e-10, edm_tol=1e-20)
    assert r.x[1] == 0.0
    assert np.allclose(r.x[[0, 2]], c[[0, 2]], atol=1e-7)


def test_hessian_errors_of_gaussian_likelihood():
    """NLL of a Gaussian mean: sigma_mean = sigma / sqrt(n)."""
    rng = np.random.default_rng(0)
    data = rng.normal(3.0, 2.0, 400)

    def nll(p):
        mu, sig = p
        r = (data - mu) / sig
        f = 0.5 * float(r @ r) + len(data) * np.log(sig)
        g = np.array([-float(r.sum()) / sig, -float(r @ r) / sig + len(data) / sig])
        return f, g
    r = minimize.bfgs(nll, np.array([0.0, 1.0]), gtol=1e-9, edm_tol=1e-18)
    err = minimize.errors(nll, r.x)
    assert abs(r.x[0] - data.mean()) < 1e-6
    assert abs(err[0] - r.x[1] / np.sqrt(len(data))) < 1e-4 * err[0]
