"""Pins of the FP64 network oracle used to check the library's training kernels: the
chain-rule gradient equals central finite differences of the loss.  CPU only."""
import numpy as np

from oracle import mlp


def _random_params(rng):
    P = np.zeros(mlp.SIZE)
    P[: mlp.NORM] = rng.normal(0, 0.2, mlp.NORM)
    P[mlp.NORM:mlp.NORM + 4] = [0.05, 0.05, 2.0, 0.025]
    P[mlp.NORM + 4:mlp.NORM + 8] = [0.0, 0.0, 0.5, 45.0]
    P[mlp.NORM + 8:mlp.NORM + 16] = rng.normal(0, 1, 8)
    P[mlp.NORM + 16:mlp.NORM + 24] = rng.uniform(0.5, 2.0, 8)
    return P


def test_gradient_matches_finite_differences():
    rng = np.random.default_rng(4)
    P = _random_params(rng)
    x = np.stack([rng.uniform(-20, 20, 16), rng.uniform(-20, 20, 16), rng.uniform(0, 1, 16), rng.uniform(5, 85, 16)], 1)
    y = rng.normal(0, 1, (16, 6))
    g = mlp.grad(P, x, y)
    idx = np.concatenate([rng.choice(np.arange(a, b), 6, replace=False) for a, b in
                          [(mlp.W1, mlp.B1), (mlp.B1, mlp.W2), (mlp.W2, mlp.B2), (mlp.B2, mlp.W3), (mlp.W3, mlp.B3),
                           (mlp.B3, mlp.W4), (mlp.W4, mlp.B4), (mlp.B4, mlp.NORM)]])
    for i in idx:
        h = 1e-6
        Pp, Pm = P.copy(), P.copy()
        Pp[i] += h
        Pm[i] -= h
        fd = (mlp.loss(Pp, x, y) - mlp.loss(Pm, x, y)) / (2 * h)
        assert abs(fd - g[i]) <= 1e-6 * max(1.0, abs(fd)), (i, fd, g[i])


def test_silu_derivative_and_unused_outputs():
    z = np.linspace(-8, 8, 101)
    h = 1e-6
    assert np.allclose(mlp.dsilu(z), (mlp.silu(z + h) - mlp.silu(z - h)) / (2 * h), atol=1e-8)
    rng = np.random.default_rng(5)
    P = _random_params(rng)
    x = rng.uniform(-1, 1, (8, 4))
    g = mlp.grad(P, x, rng.normal(0, 1, (8, 6)))
    # outputs 6 and 7 carry no loss: their output weights and biases get zero gradient
    W4 = g[mlp.W4:mlp.B4].reshape(8, 256)
    assert np.all(W4[6:] == 0) and np.all(g[mlp.B4 + 6:mlp.NORM] == 0)
