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


def test_bf16_round_values():
    """Round to nearest, ties to the even mantissa (BF16 keeps 7 explicit bits)."""
    one = 1.0
    cases = {one: one, one + 2**-8: one, one + 3 * 2**-8: one + 2 * 2**-7, one + 2**-8 + 2**-20: one + 2**-7,
             -(one + 3 * 2**-8): -(one + 2 * 2**-7), 3.0: 3.0, 2**-130: 2**-130, 0.0: 0.0}
    got = mlp.bf16_round(np.array(list(cases.keys())))
    assert np.array_equal(got, np.array(list(cases.values())))


def test_quantized_gradient_reduces_to_the_exact_one():
    """An identity quantizer gives the FP64 gradient bit for bit; BF16 storage moves it by a
    BF16-sized relative amount, no more (a rounding applied to the wrong quantity, e.g. the
    pre-activation, would still pass this, which is why the GPU test compares elementwise)."""
    rng = np.random.default_rng(5)
    dims = [16, 32, 32, 8]
    n_params = sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))
    layers = mlp.unflatten(rng.normal(0, 0.3, n_params), dims)
    x = rng.normal(0, 1, (24, dims[0]))
    t = rng.normal(0, 1, (24, dims[-1]))
    t[rng.random(t.shape) < 0.2] = np.nan
    L0, g0 = mlp.loss_and_grad(layers, x, t)
    L1, g1 = mlp.loss_and_grad(layers, x, t, quantize=lambda a: a)
    assert L0 == L1 and np.array_equal(g0, g1)
    L2, g2 = mlp.loss_and_grad(layers, x, t, quantize=mlp.bf16_round)
    assert abs(L2 / L0 - 1.0) < 2e-2
    assert 0.0 < np.linalg.norm(g2 - g0) / np.linalg.norm(g0) < 2e-2


def test_gradient_scale_bounds_the_gradient():
    """The absolute-term sums bound every gradient element, with and without BF16 storage,
    and are not vacuous (most elements are within a factor 100 of their bound)."""
    rng = np.random.default_rng(9)
    dims = [12, 20, 20, 6]
    n_params = sum(dims[i] * dims[i + 1] + dims[i + 1] for i in range(len(dims) - 1))
    layers = mlp.unflatten(rng.normal(0, 0.4, n_params), dims)
    x = rng.normal(0, 1, (32, dims[0]))
    t = rng.normal(0, 1, (32, dims[-1]))
    t[rng.random(t.shape) < 0.15] = np.nan
    for q in (None, mlp.bf16_round):
        _, g = mlp.loss_and_grad(layers, x, t, quantize=q)
        sc = mlp.gradient_scale(layers, x, t, quantize=q)
        assert np.all(np.abs(g) <= sc * (1 + 1e-12))
        assert np.median(np.abs(g) / sc) > 1e-2
