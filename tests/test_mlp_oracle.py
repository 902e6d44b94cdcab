"""Pins of the CPU reference MLP: gradients against central finite differences."""
import numpy as np
import pytest

from oracle import mlp


@pytest.mark.parametrize("seed", [0, 1])
def test_mlp_gradient_matches_finite_differences(seed):
    rng = np.random.default_rng(seed)
    dims = [6, 5, 4, 3]
    n_params = sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))
    flat = rng.normal(0, 0.7, n_params)
    x = rng.normal(0, 1, (7, dims[0]))
    t = rng.normal(0, 1, (7, dims[-1]))
    t[1, 2] = np.nan  # masked target
    t[4, 0] = np.nan
    L, g = mlp.loss_and_grad(mlp.unflatten(flat, dims), x, t)
    assert np.isfinite(L)
    h = 1e-6
    fd = np.zeros_like(flat)
    for i in range(flat.size):
        p, q = flat.copy(), flat.copy()
        p[i] += h
        q[i] -= h
        fd[i] = (mlp.loss(mlp.unflatten(p, dims), x, t) - mlp.loss(mlp.unflatten(q, dims), x, t)) / (2 * h)
    assert np.allclose(g, fd, rtol=1e-6, atol=1e-9)


def test_gelu_values():
    # GELU(0) = 0, GELU(x) -> x for large x, GELU'(0) = 1/2
    assert mlp.gelu(np.array([0.0]))[0] == 0.0
    assert abs(mlp.gelu(np.array([8.0]))[0] - 8.0) < 1e-12
    assert abs(mlp.gelu_grad(np.array([0.0]))[0] - 0.5) < 1e-15
    x = np.linspace(-3, 3, 13)
    fd = (mlp.gelu(x + 1e-6) - mlp.gelu(x - 1e-6)) / 2e-6
    assert np.allclose(mlp.gelu_grad(x), fd, atol=1e-8)
